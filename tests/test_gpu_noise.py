"""Diagonal, state-dependent noise coefficients (the section on filtering with noise
coefficients) on the device against the FP64 oracle: step-local parity of the prediction
(metric a(x)^+ of the target, 1/2 log det_+ a) and of the b(x)^-1-weighted update, with an
invertible and with a singular a(x); a whole run with restarts; and the refusal of the
configurations the library does not run."""
import numpy as np
import pytest

from synth import simulate

from ._helpers import combination_err_ok, oracle_problem, rel_err, sobol_inputs

pytestmark = pytest.mark.gpu

NOISE = {"inv": dict(u=0.7, u_kappa=0.8, u_zero=0, v=1.3, v_kappa=0.5),
         "sing": dict(u=0.9, u_kappa=0.4, u_zero=2, v=0.8, v_kappa=1.0)}


def _make(model, r, n, R, N, prec, noise, seed, restart_interval=0):
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model=model, r=r, n=n, dt=0.01, R=R, n_scales=N, precision=prec, noise=noise,
                              restart_interval=restart_interval)
    f = binding.Filter(cfg)
    poly, scr = sobol_inputs(r, seed)
    f.init_nodes(poly, scr, np.zeros(r))
    return f


@pytest.mark.parametrize("model,r,n,R,N,prec,nz", [("cubic", 3, 1500, 1.0, 2, "f32", "inv"),
                                                   ("cubic", 3, 1500, 1.0, 2, "f64", "inv"),
                                                   ("linear", 5, 2000, 0.8, 1, "f32", "sing"),
                                                   ("cubic", 40, 1024, 0.3, 2, "f32", "sing"),
                                                   ("cubic", 70, 777, 0.3, 3, "f64", "inv")])
def test_step_local_parity_with_noise_coefficients(yy_lib, model, r, n, R, N, prec, nz):
    import torch
    from oracle import filter as F
    noise = NOISE[nz]
    tol = 1e-10 if prec == "f64" else 1e-5
    f = _make(model, r, n, R, N, prec, noise, 77)
    u, _ = f.get_nodes()
    p = oracle_problem(model, r, n, 0.01, R, N, noise=noise)
    tr = simulate(model, r, 3, 0.01, seed=77, noise=noise)
    st = F.init_state(p, u, np.zeros(r))
    for k in range(2):
        _, st = F.step(p, st, tr.dy[k])
    T = np.float64 if prec == "f64" else np.float32
    lw_in = st.logw.astype(T).astype(np.float64)
    f.set_state(st.centre, st.logw.astype(T), st.lognorm, st.k)
    f.predict()
    pred, off = f.get_log_weights()
    prep = F.prepare(p, u, st.centre)
    Lj = F.kernel_lse(p, prep, lw_in)
    ref, _ = F.combine(p, Lj, lw_in, prep.mask)
    ok, kappa = combination_err_ok(pred.astype(np.float64) + off, ref, Lj, p.coef, lw_in, tol,
                                   eps=2.0 ** -53 if prec == "f64" else 2.0 ** -24)
    print(f"{model} r={r} {prec} {nz}: largest combination condition number {kappa:.1f}")
    assert ok
    f.update(torch.tensor(tr.dy[2], dtype=torch.float64, device="cuda"))
    mean, var, ess, z = f.estimate()
    lw_hat, _ = f.get_log_weights()
    rec, _ = F.step(p, F.State(u=u, centre=st.centre, logw=lw_in, lognorm=st.lognorm, k=st.k), tr.dy[2],
                    keep_logw=True)
    # the update alone: the GPU's own predicted weights through the oracle's correction
    upd = pred.astype(np.float64) + off + F.log_likelihood(p, prep.x, tr.dy[2])
    assert rel_err(lw_hat, F.normalise(upd)[1]) <= tol
    assert np.max(np.abs(mean - rec.mean) / np.maximum(1.0, np.abs(rec.mean))) <= 10 * tol
    assert abs(ess - rec.ess) <= 10 * tol * rec.ess


def test_whole_run_with_noise_coefficients_fp64(yy_lib):
    import torch
    from oracle import filter as F
    r, n, R, N, K = 4, 2048, 0.6, 2, 40
    noise = NOISE["sing"]
    f = _make("cubic", r, n, R, N, "f64", noise, 78, restart_interval=2)
    u, _ = f.get_nodes()
    p = oracle_problem("cubic", r, n, 0.01, R, N, restart_interval=2, noise=noise)
    tr = simulate("cubic", r, K, 0.01, seed=78, noise=noise)
    recs = F.run(p, F.init_state(p, u, np.zeros(r)), tr.dy)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    hist = torch.zeros((K, 2 * r + 4), dtype=torch.float64, device="cuda")
    f.run_steps(dy, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    ref = np.array([q.mean for q in recs])
    print("max |x_hat - oracle|", np.max(np.abs(h[:, :r] - ref)))
    assert np.max(np.abs(h[:, :r] - ref)) <= 1e-8


def test_unsupported_noise_configurations(yy_lib):
    from paper_2509_16896_gb300 import binding
    for prec, model in (("bf16", "cubic"), ("f32s", "cubic"), ("f32", "paper_e1")):
        cfg = binding.make_config(model=model, r=4, n=512, dt=0.01, R=0.3, n_scales=2, precision=prec,
                                  noise=NOISE["inv"])
        with pytest.raises(binding.YYError) as ei:
            binding.Filter(cfg)
        assert ei.value.code == 8   # YY_ERR_UNSUPPORTED
