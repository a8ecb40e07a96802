"""yy_weighted_moments_static, the entry point that allocates no device memory (its
scratch is a fixed device array inside the library), against the FP64 oracle's
normalisation and estimate and against the handle-based path (yy_update + yy_estimate).

It serves callers that cannot call cudaMalloc when they need the result (host
callbacks, plug-ins whose host owns all device buffers, allocation-free real-time
loops).  Calls come in pairs with different inputs, so that the shared scratch is shown
to keep nothing from the previous call that matters.  Sizes cover fewer rows than the
entry point's 120 reduction blocks (n = 1, 7, 119), a ragged count, the largest r, and
all weights -inf.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from synth import simulate

from ._helpers import sobol_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the float32 bar of the parity tests


def _call(u, lw):
    import torch
    from paper_2509_16896_gb300 import binding
    r = u.shape[1]
    out = torch.full((2 * r + 3,), float("nan"), dtype=torch.float64, device="cuda")
    binding.weighted_moments_static(u, lw, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _check_against_oracle(o, u_host, lw_host):
    """o = mean, var, ESS, LSE, weight sum of the GPU call; the oracle in float64 on the
    same float32 inputs."""
    from oracle import filter as F
    r = u_host.shape[1]
    lw64 = lw_host.astype(np.float64)
    lam, lh = F.normalise(lw64)
    mean, var, ess = F.estimate(u_host.astype(np.float64), lh)
    assert abs(o[2 * r + 1] - lam) <= TOL * max(1.0, abs(lam))
    scale = max(1.0, float(np.max(np.abs(u_host))))
    assert np.max(np.abs(o[:r] - mean)) <= TOL * scale
    assert np.all(np.abs(o[r:2 * r] - var) <= TOL * np.abs(var) + 1e-12 * scale ** 2)
    assert abs(o[2 * r] - ess) <= TOL * ess
    assert abs(o[2 * r + 2] - 1.0) <= TOL


@pytest.mark.parametrize("n,r", [(1, 3), (7, 5), (119, 33), (1000, 17), (4099, 1024)])
def test_static_scratch_matches_oracle(yy_lib, n, r):
    import torch
    rng = np.random.default_rng(n * 1000 + r)
    for call in range(2):   # two calls in a row with different inputs
        u = rng.uniform(-0.3, 0.3, size=(n, r)).astype(np.float32)
        lw = (rng.normal(scale=3.0, size=n) + 50.0 * call).astype(np.float32)
        if n > 5:
            lw[rng.choice(n, size=n // 5, replace=False)] = -np.inf   # dead nodes
        o = _call(torch.tensor(u, device="cuda"), torch.tensor(lw, device="cuda"))
        _check_against_oracle(o, u, lw)


def test_all_weights_minus_inf_reads_as_empty(yy_lib):
    import torch
    r, n = 4, 300
    u = torch.rand((n, r), dtype=torch.float32, device="cuda")
    ok = np.random.default_rng(1).normal(size=n).astype(np.float32)
    for lw in (np.full(n, -np.inf, dtype=np.float32), ok, np.full(n, -np.inf, dtype=np.float32)):
        o = _call(u, torch.tensor(lw, device="cuda"))
        if np.all(np.isneginf(lw)):
            assert np.isneginf(o[2 * r + 1]) and o[2 * r + 2] == 0.0 and o[2 * r] == 0.0
            assert np.all(o[:2 * r] == 0.0)
        else:
            _check_against_oracle(o, u.cpu().numpy(), lw)


@pytest.mark.parametrize("r,n", [(17, 1000), (1000, 4096)])
def test_static_scratch_moments_match_handle_path(yy_lib, r, n):
    import torch
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=0.3, n_scales=2, precision="f32")
    flt = binding.Filter(cfg)
    poly, scr = sobol_inputs(r, 31)
    flt.init_nodes(poly, scr, np.zeros(r))
    tr = simulate("cubic", r, 1, 0.01, seed=31)
    flt.predict()
    flt.update(torch.tensor(tr.dy[0], dtype=torch.float64, device="cuda"))
    mean, var, ess, _ = flt.estimate()
    centre, _, _ = flt.get_state()
    lw, off = flt.get_log_weights()
    assert off == 0.0
    u, _ = flt.get_nodes()

    u_dense = torch.tensor(u, device="cuda")
    u_wide = torch.zeros((n, r + 5), dtype=torch.float32, device="cuda")
    u_wide[:, :r] = u_dense
    calls = [(u_dense, torch.tensor(lw, device="cuda"), 0.0),
             (u_wide[:, :r], torch.tensor(lw + np.float32(3.7), device="cuda"), 3.7)]
    for u_dev, lw_dev, shift in calls:
        o = _call(u_dev, lw_dev)
        m_static = centre + o[:r]
        assert np.max(np.abs(m_static - mean) / np.maximum(1.0, np.abs(mean))) <= TOL
        assert np.all(np.abs(o[r:2 * r] - var) <= TOL * np.abs(var) + 1e-12)
        assert abs(o[2 * r] - ess) <= TOL * ess
        assert abs(o[2 * r + 1] - shift) <= TOL * max(1.0, shift)
        assert abs(o[2 * r + 2] - 1.0) <= TOL


def test_static_scratch_rejects_sizes_beyond_its_limit(yy_lib):
    import ctypes

    import torch
    from paper_2509_16896_gb300 import binding
    L = binding.load()
    u = torch.zeros((4, 1025), dtype=torch.float32, device="cuda")
    lw = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(2 * 1025 + 3, dtype=torch.float64, device="cuda")
    P = ctypes.c_void_p
    rc = L.yy_weighted_moments_static(P(u.data_ptr()), 4, 1025, 1025, P(lw.data_ptr()),
                                      P(out.data_ptr()), None)
    assert rc == 1   # YY_ERR_ARG: r above YY_NOALLOC_MAX_DIM, nothing launched
    rc = L.yy_weighted_moments_static(P(u.data_ptr()), 4, 8, 4, P(lw.data_ptr()), P(out.data_ptr()), None)
    assert rc == 1   # row stride shorter than a row
    rc = L.yy_weighted_moments_static(P(u.data_ptr()), 0, 8, 8, P(lw.data_ptr()), P(out.data_ptr()), None)
    assert rc == 1   # no rows
