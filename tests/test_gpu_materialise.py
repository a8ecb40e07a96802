"""The materialised schedule of the prediction (the paper's offline operator with an online
log-domain matrix-vector product): the per-scale operator built on the device once per node
set and applied at every prediction, against the FP64 oracle on the r = 100, n = 16384
workload's shape with restarts every third step (a node set serves three predictions):
step-local at 1e-5, and a whole run in which every restart makes the device rebuild the
operator (also inside a replayed CUDA graph).  The autotuner's timings and choice are
reported."""
import os

import numpy as np
import pytest

from synth import simulate

from ._helpers import oracle_problem, rel_err, sobol_inputs

pytestmark = pytest.mark.gpu


def _make(r, n, N, prec, materialise, iota, seed, stream=None):
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=0.3, n_scales=N, precision=prec,
                              restart_interval=iota, ess_frac=0.0, materialise=materialise)
    f = binding.Filter(cfg, stream=stream)
    poly, scr = sobol_inputs(r, seed)
    f.init_nodes(poly, scr, np.zeros(r))
    return f


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_materialised_prediction_step_local(yy_lib, prec):
    from oracle import filter as F
    r, n, N = 100, 16384, 2
    f = _make(r, n, N, prec, 2, 3, 2)
    u, _ = f.get_nodes()
    p = oracle_problem("cubic", r, n, 0.01, 0.3, N, restart_interval=3)
    tr = simulate("cubic", r, 3, 0.01, seed=2)
    st = F.init_state(p, u, np.zeros(r))
    for k in range(2):
        _, st = F.step(p, st, tr.dy[k], n_threads=os.cpu_count() or 1)
    f.set_state(st.centre, st.logw.astype(np.float32), st.lognorm, st.k)
    rows = np.r_[0:512, n - 512:n]
    ref, _ = F.predict(p, F.prepare(p, u, st.centre), st.logw.astype(np.float32).astype(np.float64),
                       0, n, n_threads=os.cpu_count() or 1)
    for rep in range(2):   # the first prediction builds the operator, the second reuses it
        f.predict()
        pred, off = f.get_log_weights()
        assert rel_err((pred.astype(np.float64) + off)[rows], ref[rows]) <= 1e-5, rep


@pytest.mark.parametrize("prec,r,n,N", [("f32", 7, 3001, 3), ("bf16", 33, 5002, 1), ("f32", 12, 2053, 4),
                                         ("bf16", 16, 515, 2)])
def test_materialised_prediction_ragged(yy_lib, prec, r, n, N):
    """Node counts that end inside a group of four columns and inside a block of rows, at
    every scale count: every row against the oracle, for the build and the reuse."""
    from oracle import filter as F
    f = _make(r, n, N, prec, 2, 3, 11)
    u, _ = f.get_nodes()
    p = oracle_problem("cubic", r, n, 0.01, 0.3, N, restart_interval=3)
    tr = simulate("cubic", r, 2, 0.01, seed=11)
    st = F.init_state(p, u, np.zeros(r))
    _, st = F.step(p, st, tr.dy[0], n_threads=os.cpu_count() or 1)
    f.set_state(st.centre, st.logw.astype(np.float32), st.lognorm, st.k)
    ref, _ = F.predict(p, F.prepare(p, u, st.centre), st.logw.astype(np.float32).astype(np.float64),
                       0, n, n_threads=os.cpu_count() or 1)
    for rep in range(2):
        f.predict()
        pred, off = f.get_log_weights()
        full = pred.astype(np.float64) + off
        assert np.array_equal(np.isneginf(full), np.isneginf(ref)), rep
        assert rel_err(full, ref) <= 1e-5, rep


def test_materialised_whole_run_and_graph(yy_lib):
    import torch
    from oracle import filter as F
    r, n, N, K = 100, 16384, 2, 9
    tr = simulate("cubic", r, K, 0.01, seed=2)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    f = _make(r, n, N, "f32", 2, 3, 2)
    u, _ = f.get_nodes()
    hist = torch.zeros((K, 2 * r + 4), dtype=torch.float64, device="cuda")
    f.run_steps(dy, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    p = oracle_problem("cubic", r, n, 0.01, 0.3, N, restart_interval=3)
    recs = F.run(p, F.init_state(p, u, np.zeros(r)), tr.dy, n_threads=os.cpu_count() or 1)
    ref = np.array([q.mean for q in recs])
    scale = float(np.sqrt(np.mean(tr.x ** 2)))
    print("materialised whole run: max |x_hat - oracle|", float(np.max(np.abs(h[:, :r] - ref))))
    assert np.array_equal(h[:, 2 * r + 3], np.array([1.0 if q.restarted else 0.0 for q in recs]))
    assert np.max(np.abs(h[:, :r] - ref)) <= 1e-3 * scale
    # the same steps replayed from a CUDA graph (restarts inside the graph trigger the rebuilds)
    s = torch.cuda.Stream()
    g = _make(r, n, N, "f32", 2, 3, 2, stream=s)
    hg = torch.zeros((K, 2 * r + 4), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        g.graph_capture(dy, hg)
    g.graph_launch()
    torch.cuda.synchronize()
    assert np.array_equal(hg.cpu().numpy(), h)


def test_tuner_reports_and_chooses(yy_lib):
    f = _make(100, 16384, 2, "bf16", 1, 3, 2)
    choice, (re, bu, ap) = f.tune_materialise(3, reps=3)
    print(f"r=100 n=16384 N=2: recompute {re:.3f} ms, build {bu:.3f} ms, apply {ap:.3f} ms, materialised chosen: {choice}")
    assert re > 0 and bu > 0 and ap > 0
    assert choice == int(bu + 3 * ap < 3 * re)
