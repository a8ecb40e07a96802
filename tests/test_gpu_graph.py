"""K-step runs without host round trips (yy_run_steps) and their CUDA-graph capture:
the replay must reproduce the step-by-step calls exactly."""
import numpy as np
import pytest

from synth import simulate

from ._helpers import sobol_inputs

pytestmark = pytest.mark.gpu


def _filter(prec, r=40, n=3000, N=2, stream=None):
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=0.3, n_scales=N, precision=prec,
                              restart_interval=2, ess_frac=0.5)
    flt = binding.Filter(cfg, stream=stream)
    poly, scr = sobol_inputs(r, 41)
    flt.init_nodes(poly, scr, np.zeros(r))
    return flt


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_run_steps_and_graph_match_individual_calls(yy_lib, prec):
    import torch
    r, K = 40, 6
    tr = simulate("cubic", r, 2 * K, 0.01, seed=41)
    dys = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    # reference: one call at a time, estimate read after every step
    ref = []
    f0 = _filter(prec)
    for k in range(2 * K):
        f0.predict()
        f0.update(dys[k])
        m, v, e, z = f0.estimate()
        ref.append(np.concatenate([m, v, [e, z]]))
        f0.restart(mode=0)
    ref = np.array(ref)
    # same steps through yy_run_steps
    f1 = _filter(prec)
    h1 = torch.zeros((2 * K, 2 * r + 4), dtype=torch.float64, device="cuda")
    f1.run_steps(dys, h1)
    h1 = h1.cpu().numpy()
    assert np.array_equal(h1[:, :2 * r], ref[:, :2 * r])
    assert np.array_equal(h1[:, 2 * r], ref[:, 2 * r]) and np.array_equal(h1[:, 2 * r + 2], ref[:, 2 * r + 1])
    # graph: capture K steps, replay twice on fresh increments (buffer refilled in between)
    s = torch.cuda.Stream()
    f2 = _filter(prec, stream=s)
    buf = torch.empty((K, r), dtype=torch.float64, device="cuda")
    h2 = torch.zeros((K, 2 * r + 4), dtype=torch.float64, device="cuda")
    f2.graph_capture(buf, h2)
    assert f2.graph_kernels() > 0
    out = []
    for rep in range(2):
        with torch.cuda.stream(s):
            buf.copy_(dys[rep * K:(rep + 1) * K])
            f2.graph_launch()
            out.append(h2.clone())
    torch.cuda.synchronize()
    h2all = torch.cat(out).cpu().numpy()
    assert np.array_equal(h2all, h1)


def test_graph_needs_a_created_stream(yy_lib):
    import torch
    from paper_2509_16896_gb300 import binding
    f = _filter("f32", stream=torch.cuda.default_stream())
    with pytest.raises(binding.YYError) as ei:
        f.graph_capture(torch.zeros((2, 40), dtype=torch.float64, device="cuda"))
    assert ei.value.code == 7
