"""Two-pass BF16 screen of the prediction: a first pass over the first 64 k coordinates
(restricted to them |u_i - u_s| is still a lower bound of the distance), tiles whose warps
keep many candidates screened again over all coordinates.  Every first-pass length must give
the FP32 form's predictions to float32 rounding; short first passes must actually rescreen;
the device-side choice of the length must stay in range over a run with restarts."""
import numpy as np
import pytest

from synth import simulate

from ._helpers import rel_err, sobol_inputs

pytestmark = pytest.mark.gpu


def _filter(r, n, N, prec, prefix=0, restart_interval=0, screen="bf16"):
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=0.3, n_scales=N, precision=prec,
                              restart_interval=restart_interval, screen_prefix=prefix, screen_type=screen)
    return binding.Filter(cfg)


@pytest.mark.parametrize("screen", ["bf16", "fp8"])
@pytest.mark.parametrize("r,n,N", [(1000, 4096, 3), (300, 3000, 2), (130, 2500, 2)])
def test_every_first_pass_length_matches_fp32_path(yy_lib, r, n, N, screen):
    import torch
    poly, scr = sobol_inputs(r, 31)
    tr = simulate("cubic", r, 3, 0.01, seed=31)
    ref = _filter(r, n, N, "f32")
    ref.init_nodes(poly, scr, np.zeros(r))
    from paper_2509_16896_gb300 import binding
    for k in range(2):
        ref.predict()
        ref.update(torch.tensor(tr.dy[k], dtype=torch.float64, device="cuda"))
    # a restart's Gaussian weights spread over hundreds of nats at high r
    ref.restart(binding.RESTART_FORCE)
    centre, lognorm, step = ref.get_state()
    logw, off = ref.get_log_weights()
    assert off == 0.0   # normalised after a restart
    spread = np.ptp(logw[np.isfinite(logw)])
    ref.predict()
    a, a_off = ref.get_log_weights()
    a = a.astype(np.float64) + a_off
    # stages of 64 (BF16 operands) or 128 (FP8 operands) coordinates
    nk = (r + 63) // 64 if screen == "bf16" else ((r + 63) // 64 * 64 + 127) // 128
    n_pad = (n + 255) // 256 * 256
    seen = {}
    for prefix in sorted({1, 2, max(1, nk // 2), nk, 0}):
        flt = _filter(r, n, N, "bf16", prefix=prefix, screen=screen)
        flt.init_nodes(poly, scr, np.zeros(r))
        flt.set_state(centre, logw.astype(np.float32), lognorm, step)
        flt.predict()
        b, b_off = flt.get_log_weights()
        assert rel_err(b.astype(np.float64) + b_off, a) <= 2e-6, (prefix, spread)
        last, nxt, tiles, resc = flt.screen()
        # the screen covers the upper block triangle: target tile a (128 rows) against the
        # source tiles (256) from the one holding its first row on
        nst = n_pad // 256
        assert tiles == sum(nst - a // 2 for a in range(n_pad // 128))
        assert 0 <= resc <= tiles
        assert 1 <= last <= nk and 1 <= nxt <= nk
        if prefix == nk:
            assert resc == 0 and last == nk
            if r == 1000:   # a sound Gram product screens out nearly every pair at full length
                assert flt.counters()[1] < 0.001 * n * n
        if prefix > 0:
            assert last == nxt == min(prefix, nk)   # a fixed length is kept
        seen[prefix] = resc
    if r == 1000 and screen == "bf16":
        # 64 coordinates cannot separate pairs whose weights differ by a hundred nats or more
        assert spread > 100 and seen[1] > 0


def test_adaptive_first_pass_over_a_run(yy_lib):
    """r = 1000 with restarts every second step: the chosen length stays in [1, nk], and the
    run's estimates match the FP32 form's run on the same data."""
    import torch
    r, n, N, K = 1000, 4096, 3, 10
    poly, scr = sobol_inputs(r, 32)
    tr = simulate("cubic", r, K, 0.01, seed=32)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    hist = {}
    lens = []
    for prec in ("f32", "bf16"):
        flt = _filter(r, n, N, prec, restart_interval=2)
        flt.init_nodes(poly, scr, np.zeros(r))
        h = torch.zeros((K, 2 * r + 4), dtype=torch.float64, device="cuda")
        for k in range(K):
            flt.run_steps(dy[k:k + 1], h[k:k + 1])
            if prec == "bf16":
                lens.extend(flt.screen()[:2])
        torch.cuda.synchronize()
        hist[prec] = h.cpu().numpy()
    nk = (r + 63) // 64
    assert all(1 <= v <= nk for v in lens)
    a, b = hist["f32"], hist["bf16"]
    assert np.array_equal(a[:, 2 * r + 3], b[:, 2 * r + 3])          # same restart steps
    assert np.max(np.abs(a[:, :r] - b[:, :r])) <= 1e-4               # posterior means
    assert np.max(np.abs(a[:, r:2 * r] - b[:, r:2 * r]) / a[:, r:2 * r]) <= 1e-3   # variances
