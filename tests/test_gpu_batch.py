"""Batches of ragged filters in one launch per pass (include/yy.h, batch section): every
member must reproduce its own single-filter run, the captured graph must reproduce the
step calls, and every schedule the autotuner can pick must give the same answer."""
import numpy as np
import pytest

from synth import simulate

from ._helpers import sobol_inputs

pytestmark = pytest.mark.gpu

# (model, r, n, seed): ragged shapes, not multiples of any tile
MEMBERS = [("cubic", 10, 2048, 51), ("linear", 33, 3000, 52), ("cubic", 70, 1500, 53),
           ("linear", 130, 4100, 54), ("cubic", 17, 2600, 55), ("cubic", 64, 999, 56)]


def _cfgs(prec):
    from paper_2509_16896_gb300 import binding
    return [binding.make_config(model=m, r=r, n=n, dt=0.01, R=0.3, n_scales=2, precision=prec,
                                restart_interval=2, ess_frac=0.5) for (m, r, n, _) in MEMBERS]


def _inputs(K):
    import torch
    dys = [simulate(m, r, K, 0.01, seed=s).dy for (m, r, n, s) in MEMBERS]
    return dys, torch.tensor(np.concatenate(dys, axis=1), dtype=torch.float64, device="cuda")


def _batch(prec, cfgs=None):
    from paper_2509_16896_gb300 import binding
    bt = binding.Batch(cfgs or _cfgs(prec))
    for b, (m, r, n, s) in enumerate(MEMBERS):
        poly, scr = sobol_inputs(r, s)
        bt.filters[b].init_nodes(poly, scr, np.zeros(r))
    return bt


@pytest.mark.parametrize("prec", ["bf16", "f32"])
def test_batch_matches_single_filters(yy_lib, prec):
    import torch
    from paper_2509_16896_gb300 import binding
    K = 5
    dys, dy_all = _inputs(K)
    bt = _batch(prec)
    hist = torch.zeros((K, bt.H), dtype=torch.float64, device="cuda")
    bt.run_steps(dy_all, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    for b, ((m, r, n, s), cfg) in enumerate(zip(MEMBERS, _cfgs(prec))):
        f = binding.Filter(cfg)
        poly, scr = sobol_inputs(r, s)
        f.init_nodes(poly, scr, np.zeros(r))
        hs = torch.zeros((K, 2 * r + 4), dtype=torch.float64, device="cuda")
        f.run_steps(torch.tensor(dys[b], dtype=torch.float64, device="cuda"), hs)
        hs = hs.cpu().numpy()
        hb = h[:, bt.hist_off[b]:bt.hist_off[b + 1]]
        # same kernels, different reduction split (16 blocks per member instead of 304)
        assert np.max(np.abs(hb[:, :r] - hs[:, :r]) / np.maximum(1.0, np.abs(hs[:, :r]))) <= 1e-5, b
        assert np.all(np.abs(hb[:, r:2 * r] - hs[:, r:2 * r]) <= 1e-5 * np.abs(hs[:, r:2 * r]) + 1e-12), b
        assert np.allclose(hb[:, 2 * r], hs[:, 2 * r], rtol=1e-5), b
        assert np.array_equal(hb[:, 2 * r + 3], hs[:, 2 * r + 3]), b
        # the borrowed handle reports the same state as the batch history
        mean, var, ess, z = bt.filters[b].estimate()
        assert np.allclose(mean, hb[-1, :r], rtol=0, atol=0)


def test_batch_graph_replays_run_steps(yy_lib):
    import torch
    K = 4
    _, dy_all = _inputs(2 * K)
    a = _batch("bf16")
    ha = torch.zeros((2 * K, a.H), dtype=torch.float64, device="cuda")
    a.run_steps(dy_all, ha)
    torch.cuda.synchronize()
    g = _batch("bf16")
    buf = torch.empty((K, g.M), dtype=torch.float64, device="cuda")
    hg = torch.zeros((K, g.H), dtype=torch.float64, device="cuda")
    g.graph_capture(buf, hg)
    assert g.graph_kernels() > 0
    out = []
    with torch.cuda.stream(g.stream):
        for rep in range(2):
            buf.copy_(dy_all[rep * K:(rep + 1) * K])
            g.graph_launch()
            out.append(hg.clone())
    torch.cuda.synchronize()
    assert np.array_equal(torch.cat(out).cpu().numpy(), ha.cpu().numpy())


def test_every_schedule_gives_the_same_prediction(yy_lib, tmp_path):
    import torch
    K = 2
    _, dy_all = _inputs(K)
    ref = None
    for bn, grid in [(256, 148), (128, 296), (256, 40), (128, 7)]:
        bt = _batch("bf16")
        bt.set_schedule(bn, grid)
        hist = torch.zeros((K, bt.H), dtype=torch.float64, device="cuda")
        bt.run_steps(dy_all, hist)
        torch.cuda.synchronize()
        h = hist.cpu().numpy()
        if ref is None:
            ref = h
        else:
            assert np.max(np.abs(h - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-6
    bt = _batch("bf16")
    cache = str(tmp_path / "tune.txt")
    bn, grid = bt.autotune(cache, reps=2)
    assert bn in (128, 256) and 1 <= grid <= 1024
    assert bt.schedule() == (bn, grid)
    routing = bt.routing()
    bt2 = _batch("bf16")
    assert bt2.autotune(cache, reps=2) == (bn, grid)   # cached choice reused
    assert np.array_equal(bt2.routing(), routing)
    # the tuned batch (some members possibly on the FP32 form) gives the same answer
    hist = torch.zeros((K, bt.H), dtype=torch.float64, device="cuda")
    bt.run_steps(dy_all, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    assert np.max(np.abs(h - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-5
