"""The tensor-core screen where many pairs survive it, at a size where its whole machinery
runs: n = 32768 nodes (target tiles split over two source ranges, merged by k_tc_merge),
r = 80 > 64 (symmetric blocks: the column direction adds into the per-node log-sum-exp
words by compare-and-swap), and a box narrow enough (R = 0.16) that tens of thousands of
pairs are within reach of the kernel and are evaluated exactly, with first-pass tiles
escalated to a full-coordinate second pass.  Sampled blocks of target rows, each against
all sources, must match the FP64 oracle within the float32 bar, for both operand types of
the screen and with the device-chosen first pass."""
import os

import numpy as np
import pytest

from synth import simulate, sobol_poly_params, sobol_scramble_params

from ._helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("r,n,R,N,screen", [(80, 32768, 0.16, 2, "bf16"), (80, 32768, 0.16, 2, "fp8"),
                                            (72, 40000, 0.17, 3, "bf16")])
def test_many_exact_pairs_match_oracle(yy_lib, r, n, R, N, screen):
    import torch
    from oracle import filter as F
    from paper_2509_16896_gb300 import binding
    seed = 17
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=R, n_scales=N, precision="bf16",
                              restart_interval=2, ess_frac=0.5, screen_type=screen)
    stream = torch.cuda.Stream()
    flt = binding.Filter(cfg, stream=stream)
    flt.init_nodes(sobol_poly_params(r, seed), sobol_scramble_params(r, seed), np.zeros(r))
    tr = simulate("cubic", r, 3, 0.01, seed=seed)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        flt.run_steps(dy)
    torch.cuda.synchronize()
    centre, _, _ = flt.get_state()
    _, half = flt.get_box()
    logw, off = flt.get_log_weights()
    assert off == 0.0
    u, mask = flt.get_nodes()
    flt.predict()
    pred, poff = flt.get_log_weights()
    pred = pred.astype(np.float64) + poff
    clamps, exact = flt.counters()
    last, nxt, tiles, resc = flt.screen()
    print(f"r={r} n={n} {screen}: exact pairs {exact}, tiles {tiles}, rescreened {resc}, first pass {last}")
    assert exact >= 1000, exact                       # the exact-pair path really ran
    assert not np.any(np.isnan(pred)) and np.array_equal(np.isneginf(pred), mask)
    p = F.Problem(model="cubic", r=r, n=n, dt=0.01, R=half.copy(), n_scales=N)
    prep = F.prepare(p, u, centre, half)
    lw = logw.astype(np.float64)
    rng = np.random.Generator(np.random.Philox(key=777 + r))
    # row blocks at the start, the end (ragged tail) and inside: 24 rows each
    starts = sorted(set([0, n - 24, min(n - 24, 16384 - 12)] + [int(s) for s in rng.integers(0, n - 24, size=5)]))
    threads = os.cpu_count() or 1
    worst = 0.0
    for s0 in starts:
        ref, _ = F.predict(p, prep, lw, s0, s0 + 24, n_threads=threads)
        worst = max(worst, rel_err(pred[s0:s0 + 24], ref))
    assert worst <= TOL, worst
