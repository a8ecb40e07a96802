"""One filter with its target rows split across shards, each shard a handle on the same GPU
(the exchange that several devices would do by all-gather done here by copies): every
step's estimate, normaliser, ESS and log-weights of the sharded filter must match the
whole filter within the float32 bar (1e-5 relative; FP64 1e-10), through restarts.  The
shards screen their own target tiles against every source tile while the whole filter
uses the symmetric screen, so the tensor-core cases also check that the two schedules
agree."""
import numpy as np
import pytest

from synth import simulate

from ._helpers import rel_err, sobol_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,r,n,N,G", [("bf16", 100, 4096, 2, 2), ("f32", 20, 3000, 2, 2), ("f64", 3, 1024, 2, 2),
                                          ("bf16", 1000, 2048, 3, 2), ("bf16", 40, 4096, 2, 4), ("f32s", 64, 2048, 2, 2)])
def test_shards_match_whole_filter(yy_lib, prec, r, n, N, G):
    import torch
    from paper_2509_16896_gb300 import binding
    tol = 1e-10 if prec == "f64" else 1e-5
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=0.3, n_scales=N, precision=prec,
                              restart_interval=2, ess_frac=0.5)
    poly, scr = sobol_inputs(r, 57)

    def make():
        f = binding.Filter(cfg)
        f.init_nodes(poly, scr, np.zeros(r))
        return f

    whole = make()
    shards = []
    for g in range(G):
        f = make()
        f.set_shard(g, G)
        shards.append(f)
    chunk = shards[0].shard_rows()[1]
    assert all(s.shard_rows() == (g * chunk, chunk) for g, s in enumerate(shards))
    dt = torch.float64 if prec == "f64" else torch.float32
    K = 6
    tr = simulate("cubic", r, K, 0.01, seed=57)
    dys = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    for k in range(K):
        whole.predict()
        whole.update(dys[k])
        mw, vw, ew, zw = whole.estimate()
        lw_w, _ = whole.get_log_weights()
        rows = [torch.empty(chunk, dtype=dt, device="cuda") for _ in range(G)]
        recs = torch.empty((G, 2 * r + 4), dtype=torch.float64, device="cuda")
        for g, s in enumerate(shards):
            s.predict()
            s.update_shard(dys[k], rows[g], recs[g])
        torch.cuda.synchronize()
        rows_all = torch.cat(rows)
        for s in shards:
            s.merge_shards(rows_all, recs, G)
        for g, s in enumerate(shards):
            m, v, e, z = s.estimate()
            assert np.max(np.abs(m - mw) / np.maximum(1.0, np.abs(mw))) <= tol, (k, g)
            assert np.all(np.abs(v - vw) <= tol * np.abs(vw) + 1e-12), (k, g)
            assert abs(e - ew) <= tol * ew, (k, g)
            assert abs(z - zw) <= tol * max(1.0, abs(zw)), (k, g)
            lw, off = s.get_log_weights()
            assert off == 0.0
            assert rel_err(lw, lw_w) <= tol, (k, g)
        did = whole.restart(mode=0, report=True)
        for s in shards:
            assert s.restart(mode=0, report=True) == did


def test_shard_calls_are_checked(yy_lib):
    import torch
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model="cubic", r=8, n=1000, dt=0.01, R=0.3, n_scales=2, precision="f32")
    f = binding.Filter(cfg)
    poly, scr = sobol_inputs(8, 3)
    f.init_nodes(poly, scr, np.zeros(8))
    with pytest.raises(binding.YYError):
        f.set_shard(0, 3)          # n_pad = 1024 is not a multiple of 256 x 3
    f.set_shard(1, 2)
    f.predict()
    dy = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.YYError) as ei:
        f.update(dy)               # a shard updates with yy_update_shard
    assert ei.value.code == 7
    rows = torch.empty(512, dtype=torch.float32, device="cuda")
    rec = torch.empty(20, dtype=torch.float64, device="cuda")
    f.update_shard(dy, rows, rec)
    with pytest.raises(binding.YYError):
        f.restart(mode=0)          # the step is not merged yet
    with pytest.raises(binding.YYError):
        f.merge_shards(torch.empty(1024, device="cuda"), rec.view(1, -1), 1)   # wrong shard count
