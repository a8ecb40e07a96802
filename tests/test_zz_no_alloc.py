"""yy_weighted_moments_static, the entry point that allocates no device memory (its
scratch is a fixed device array inside the library), against the handle-based path
(yy_update + yy_estimate) on the same log-weights and nodes.

It serves callers that cannot call cudaMalloc when they need the result (host
callbacks, plug-ins whose host owns all device buffers, allocation-free real-time
loops).  Two calls in a row, with different inputs, check that the shared scratch keeps
nothing from the previous call that matters.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from synth import simulate

from ._helpers import sobol_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5   # the float32 bar of the parity tests


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
        out = torch.full((2 * r + 3,), float("nan"), dtype=torch.float64, device="cuda")
        binding.weighted_moments_static(u_dev, lw_dev, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
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
