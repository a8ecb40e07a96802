"""Parity at full workload sizes in the configuration the bench times: the cubic sensor with
r = 1000, n = 65536 scrambled Sobol nodes, N = 3 bandwidths (FP8 screen operands), and with
r = 100, n = 16384, N = 2 (BF16 screen operands), the device-chosen first pass, steps
replayed as one CUDA graph.  The oracle cannot predict all 65536
rows, so it predicts sampled blocks of target rows (each against all sources) from the
exact state the GPU holds after the graph, and the GPU prediction from that state must
agree there within the float32 tolerance; the whole-vector properties (no NaN, -inf
exactly at masked nodes, finite elsewhere, the estimate inside the box) are checked at
every node."""
import os

import numpy as np
import pytest

from synth import WORKLOADS, simulate, sobol_poly_params, sobol_scramble_params

from ._helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("name", ["cubic_r1000_n65536", "cubic_r100_n16384"])
def test_full_size_sampled_rows_match_oracle(yy_lib, name):
    import torch
    from oracle import filter as F
    from paper_2509_16896_gb300 import binding
    w = WORKLOADS[name]
    W, K = 3, 4
    cfg = binding.config_from_workload(w, precision="bf16")
    stream = torch.cuda.Stream()
    flt = binding.Filter(cfg, stream=stream)
    flt.init_nodes(sobol_poly_params(w.r, w.seed), sobol_scramble_params(w.r, w.seed), np.zeros(w.r))
    tr = simulate(w.model, w.r, W + K, w.dt, seed=w.seed)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    hist = torch.zeros((K, 2 * w.r + 4), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        flt.run_steps(dy[:W])
        flt.graph_capture(dy[W:W + K], hist)
    flt.graph_launch()
    torch.cuda.synchronize()
    # the state after the graph
    centre, lognorm, step = flt.get_state()
    _, half = flt.get_box()
    logw, off = flt.get_log_weights()
    assert off == 0.0
    u, mask = flt.get_nodes()
    h = hist.cpu().numpy()
    assert np.all(np.isfinite(h[:, :2 * w.r + 3]))
    assert np.all(np.abs(h[:, :w.r] - centre[None, :]) <= 2 * half[None, :] + 1.0)
    # prediction from it on the GPU (the same kernel and first-pass controller as the graph)
    flt.predict()
    pred, poff = flt.get_log_weights()
    pred = pred.astype(np.float64) + poff
    assert not np.any(np.isnan(pred))
    assert np.array_equal(np.isneginf(pred), mask)
    assert np.all(np.isfinite(pred[~mask]))
    # oracle on sampled blocks of target rows, each against all sources
    p = F.Problem(model=w.model, r=w.r, n=w.n, dt=w.dt, R=half.copy(), n_scales=w.n_scales,
                  model_a=w.model_a)
    prep = F.prepare(p, u, centre, half)
    assert np.array_equal(prep.mask, mask)
    lw = logw.astype(np.float64)
    rng = np.random.Generator(np.random.Philox(key=20251))
    starts = sorted(set([0, w.n - 24] + [int(s) for s in rng.integers(0, w.n - 24, size=4)]))
    threads = os.cpu_count() or 1
    worst = 0.0
    for s0 in starts:
        ref, _ = F.predict(p, prep, lw, s0, s0 + 24, n_threads=threads)
        worst = max(worst, rel_err(pred[s0:s0 + 24], ref))
    assert worst <= TOL, worst
