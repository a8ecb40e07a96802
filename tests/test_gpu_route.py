"""Routing of a BF16 filter's prediction between the tensor-core screen and the plain
float32 form (yy_set_route, yy_tune_route): both routes against the FP64 oracle on every
row, the plain route against a float32 filter on the same state, whole runs with restarts
on the plain route against the float32 filter (the restarts keep the stored drift current),
and the tuner's choice against its own timings on a workload each form wins."""
import os

import numpy as np
import pytest

from synth import simulate

from ._helpers import oracle_problem, rel_err, sobol_inputs

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


def _make(model, r, n, N, prec, seed, restart_interval=0):
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model=model, r=r, n=n, dt=0.01, R=0.3, n_scales=N, precision=prec,
                              restart_interval=restart_interval, ess_frac=0.0)
    f = binding.Filter(cfg)
    poly, scr = sobol_inputs(r, seed)
    f.init_nodes(poly, scr, np.zeros(r))
    return f


def _oracle_state(model, r, n, N, u, seed):
    from oracle import filter as F
    p = oracle_problem(model, r, n, 0.01, 0.3, N)
    tr = simulate(model, r, 2, 0.01, seed=seed + 100)
    st = F.init_state(p, u, np.zeros(r))
    for k in range(2):
        _, st = F.step(p, st, tr.dy[k], n_threads=THREADS)
    return p, st


def _predict(f):
    f.predict()
    lw, off = f.get_log_weights()
    return lw.astype(np.float64) + off


@pytest.mark.parametrize("model,r,n,N,seed", [("cubic", 40, 3001, 2, 21), ("paper_e1", 100, 2048, 2, 13)])
def test_both_routes_match_oracle_and_float32(yy_lib, model, r, n, N, seed):
    from oracle import filter as F
    bf = _make(model, r, n, N, "bf16", seed)
    f32 = _make(model, r, n, N, "f32", seed)
    u, _ = bf.get_nodes()
    p, st = _oracle_state(model, r, n, N, u, seed)
    lw32 = st.logw.astype(np.float32)
    for f in (bf, f32):
        f.set_state(st.centre, lw32, st.lognorm, st.k)
    ref, _ = F.predict(p, F.prepare(p, u, st.centre), lw32.astype(np.float64), n_threads=THREADS)
    bf.set_route(True)
    plain = _predict(bf)
    assert rel_err(plain, ref) <= 1e-5
    # the float32 filter runs the same form, with its source range split across blocks
    assert rel_err(plain, _predict(f32)) <= 2e-6
    bf.set_state(st.centre, lw32, st.lognorm, st.k)   # the route changes between steps only
    bf.set_route(False)
    assert rel_err(_predict(bf), ref) <= 1e-5


@pytest.mark.parametrize("model,r,n,N,seed", [("cubic", 30, 4096, 2, 5), ("paper_e1", 20, 1500, 2, 6)])
def test_plain_route_run_with_restarts_follows_float32(yy_lib, model, r, n, N, seed):
    """Restarts move the nodes; the plain route reads the drift the preparation pass stores,
    so a stale drift would show here as a departure from the float32 filter."""
    import torch
    K = 6
    tr = simulate(model, r, K, 0.01, seed=seed)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    hists = []
    for prec in ("bf16", "f32"):
        f = _make(model, r, n, N, prec, seed, restart_interval=2)
        if prec == "bf16":
            f.set_route(True)
        h = torch.zeros((K, 2 * r + 4), dtype=torch.float64, device="cuda")
        f.run_steps(dy, h)
        torch.cuda.synchronize()
        hists.append(h.cpu().numpy())
    hb, hf = hists
    assert np.array_equal(hb[:, 2 * r + 3], hf[:, 2 * r + 3])          # same restart steps
    assert np.any(hb[:, 2 * r + 3] == 1.0)
    mean_b, mean_f = hb[:, :r], hf[:, :r]
    assert np.max(np.abs(mean_b - mean_f) / np.maximum(1.0, np.abs(mean_f))) <= 1e-5


def test_tuner_keeps_the_faster_form(yy_lib):
    from oracle import filter as F
    # the screen proves nearly every pair negligible: it wins by a wide margin
    f = _make("cubic", 100, 16384, 2, "bf16", 2)
    before = f.get_log_weights()
    route, (scr, pl) = f.tune_route(3)
    print(f"cubic r=100 n=16384: screened {scr:.3f} ms, plain {pl:.3f} ms, route {route}")
    assert route == int(pl < scr) and route == 0
    after = f.get_log_weights()
    assert np.array_equal(before[0], after[0]) and before[1] == after[1]
    # the large-scale model's weights spread over many nats: nearly every pair survives the
    # screen, and the plain form wins
    r, n, N, seed = 100, 2048, 2, 13
    g = _make("paper_e1", r, n, N, "bf16", seed)
    u, _ = g.get_nodes()
    p, st = _oracle_state("paper_e1", r, n, N, u, seed)
    lw32 = st.logw.astype(np.float32)
    g.set_state(st.centre, lw32, st.lognorm, st.k)
    route, (scr, pl) = g.tune_route(3)
    print(f"paper_e1 r=100 n=2048: screened {scr:.3f} ms, plain {pl:.3f} ms, route {route}")
    assert route == int(pl < scr) and route == 1
    ref, _ = F.predict(p, F.prepare(p, u, st.centre), lw32.astype(np.float64), n_threads=THREADS)
    assert rel_err(_predict(g), ref) <= 1e-5


def test_route_calls_are_checked(yy_lib):
    import torch
    from paper_2509_16896_gb300 import binding
    f32 = _make("cubic", 8, 1000, 2, "f32", 3)
    with pytest.raises(binding.YYError) as ei:
        f32.set_route(True)
    assert ei.value.code == 8
    with pytest.raises(binding.YYError) as ei:
        f32.tune_route(1)
    assert ei.value.code == 8
    bf = _make("cubic", 8, 1000, 2, "bf16", 3)
    bf.predict()
    with pytest.raises(binding.YYError) as ei:
        bf.set_route(True)            # between a prediction and its update
    assert ei.value.code == 7
    bf.update(torch.zeros(8, dtype=torch.float64, device="cuda"))
    bf.set_route(True)
