"""Checkpoint/resume and failure detection, in forms that fault nothing.

Resume: a run stopped after k steps, its state read with yy_get_state / yy_get_log_weights
and written into a fresh handle with yy_set_state, continues bit for bit like the run that
never stopped (FP32 form, and the tensor-core screen with a fixed first pass; the
adaptive first-pass controller's history is not part of the state, so with it results
after a resume agree only within float32 rounding).

Timeout: every pipeline wait of the tensor-core prediction kernel is bounded.  With the
limit set to a nanosecond a wait runs out on the first launch; the kernel must record
YY_ERR_TIMEOUT (read by yy_estimate), drain its own copies and tensor-core work and return,
leaving the context usable: a fresh handle then runs a clean step."""
import numpy as np
import pytest

from synth import simulate

from ._helpers import sobol_inputs

pytestmark = pytest.mark.gpu


def _filter(prec, r, n, seed, prefix=0):
    import torch
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=0.3, n_scales=2, precision=prec,
                              restart_interval=2, ess_frac=0.5, screen_prefix=prefix)
    flt = binding.Filter(cfg, stream=torch.cuda.Stream())
    poly, scr = sobol_inputs(r, seed)
    flt.init_nodes(poly, scr, np.zeros(r))
    return flt


@pytest.mark.parametrize("prec,r,n,prefix", [("f32", 20, 3000, 0), ("bf16", 130, 2048, 1), ("bf16", 40, 4096, 1)])
def test_resume_from_checkpoint_is_bit_exact(yy_lib, prec, r, n, prefix):
    import torch
    K1, K2, seed = 5, 7, 41
    tr = simulate("cubic", r, K1 + K2, 0.01, seed=seed)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    a = _filter(prec, r, n, seed, prefix)
    full = torch.zeros((K1 + K2, 2 * r + 4), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(a.stream):
        a.run_steps(dy, full)
    torch.cuda.synchronize()
    b = _filter(prec, r, n, seed, prefix)
    with torch.cuda.stream(b.stream):
        b.run_steps(dy[:K1])
    torch.cuda.synchronize()
    centre, lognorm, step = b.get_state()
    logw, off = b.get_log_weights()
    assert off == 0.0 and step == K1
    del b
    c = _filter(prec, r, n, seed, prefix)          # the resumed run: a fresh handle
    c.set_state(centre, logw, lognorm, step)
    rest = torch.zeros((K2, 2 * r + 4), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(c.stream):
        c.run_steps(dy[K1:], rest)
    torch.cuda.synchronize()
    assert np.array_equal(rest.cpu().numpy(), full[K1:].cpu().numpy())


def test_device_wait_limit_reports_timeout_and_context_survives(yy_lib):
    import torch
    from paper_2509_16896_gb300 import binding
    r, n, seed = 256, 4096, 43
    tr = simulate("cubic", r, 2, 0.01, seed=seed)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.YYError):
        _filter("bf16", r, n, seed).set_wait_limit(0.0)      # a limit must be positive
    f = _filter("bf16", r, n, seed)
    f.set_wait_limit(1e-9)
    with torch.cuda.stream(f.stream):
        f.predict()
        f.update(dy[0])
    with pytest.raises(binding.YYError) as ei:
        f.estimate()
    assert ei.value.code == 6   # YY_ERR_TIMEOUT
    torch.cuda.synchronize()    # the kernel returned: the stream drains
    del f
    g = _filter("bf16", r, n, seed)                           # default limit
    with torch.cuda.stream(g.stream):
        g.predict()
        g.update(dy[0])
    mean, var, ess, z = g.estimate()                          # YY_OK
    assert np.all(np.isfinite(mean)) and ess >= 1.0
