"""Halton and Faure node sets on the device (yy_init_nodes_lds) against the oracle:
coordinates and boundary mask bit for bit, and a filter step on those nodes within the
float32 bar (step-local: the GPU is fed the oracle's state)."""
import numpy as np
import pytest

from synth import simulate

from ._helpers import combination_err_ok, oracle_problem

pytestmark = pytest.mark.gpu


def _filter(kind, model, r, n, R, N, prec):
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model=model, r=r, n=n, dt=0.01, R=R, n_scales=N, precision=prec)
    f = binding.Filter(cfg)
    f.init_nodes_lds(kind, np.zeros(r))
    return f


@pytest.mark.parametrize("kind,r,n,R", [("halton", 1, 700, 4.0), ("halton", 3, 1000, 2.0), ("halton", 9, 4097, 0.5),
                                        ("faure", 2, 1000, 3.0), ("faure", 5, 3125, 1.0), ("faure", 12, 2000, 0.4)])
def test_lds_nodes_bit_exact(yy_lib, kind, r, n, R):
    from oracle import filter as F, lds
    f = _filter(kind, "cubic", r, n, R, 2, "f32")
    u, mask = f.get_nodes()
    ref = lds.nodes(kind, n, r, np.full(r, R))
    assert np.array_equal(u.view(np.uint32), ref.view(np.uint32))
    assert np.array_equal(mask, F.boundary_mask(ref, np.full(r, R)))


@pytest.mark.parametrize("kind,model,r,n,R,N,prec", [("halton", "cubic", 2, 2048, 3.0, 2, "f32"),
                                                     ("halton", "linear", 3, 1500, 2.0, 1, "bf16"),
                                                     ("faure", "cubic", 4, 2401, 1.0, 3, "f32"),
                                                     ("faure", "paper_e1", 7, 1000, 0.3, 2, "f64")])
def test_step_on_lds_nodes_matches_oracle(yy_lib, kind, model, r, n, R, N, prec):
    import torch
    from oracle import filter as F
    tol = 1e-10 if prec == "f64" else 1e-5
    f = _filter(kind, model, r, n, R, N, prec)
    u, _ = f.get_nodes()
    p = oracle_problem(model, r, n, 0.01, R, N)
    tr = simulate(model, r, 3, 0.01, seed=31)
    st = F.init_state(p, u, np.zeros(r))
    for k in range(2):
        _, st = F.step(p, st, tr.dy[k])
    T = np.float64 if prec == "f64" else np.float32
    f.set_state(st.centre, st.logw.astype(T), st.lognorm, st.k)
    f.predict()
    pred, off = f.get_log_weights()
    prep = F.prepare(p, u, st.centre)
    lw_in = st.logw.astype(T).astype(np.float64)
    Lj = F.kernel_lse(p, prep, lw_in)
    ref, _ = F.combine(p, Lj, lw_in, prep.mask)
    # sparse low-dimensional node sets make the N >= 2 combination (with its negative
    # coefficients) ill-conditioned in places: the float32 bar grows with its condition number
    ok, kappa = combination_err_ok(pred.astype(np.float64) + off, ref, Lj, p.coef, lw_in, tol,
                                   eps=2.0 ** -53 if prec == "f64" else 2.0 ** -24)
    print(f"{kind} r={r} n={n} N={N} {prec}: largest combination condition number {kappa:.1f}")
    assert ok
    f.update(torch.tensor(tr.dy[2], dtype=torch.float64, device="cuda"))
    mean, var, ess, z = f.estimate()
    rec, _ = F.step(p, F.State(u=u, centre=st.centre, logw=st.logw.astype(T).astype(np.float64),
                               lognorm=st.lognorm, k=st.k), tr.dy[2])
    assert np.max(np.abs(mean - rec.mean) / np.maximum(1.0, np.abs(rec.mean))) <= tol
    assert abs(ess - rec.ess) <= tol * rec.ess


def test_lds_nodes_refuse_the_learned_restart(yy_lib):
    from paper_2509_16896_gb300 import binding
    f = _filter("halton", "cubic", 3, 500, 1.0, 2, "f32")
    net = binding.MLP(3, 16, max_batch=4)
    with pytest.raises(binding.YYError) as ei:
        f.set_restart_mlp(net)
    assert ei.value.code == 8   # YY_ERR_UNSUPPORTED
    with pytest.raises(binding.YYError):
        f.sobol_bits(0, 4)
