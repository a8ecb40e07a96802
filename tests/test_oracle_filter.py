"""Pins for the oracle's correction, normalisation, estimate, restart and metrics."""
import math

import numpy as np
import pytest

from oracle import filter as F, kalman, metrics, sobol
from synth import simulate, sobol_poly_params, sobol_scramble_params


def _problem(model="cubic", r=3, n=64, R=0.5, N=2, **kw):
    return F.Problem(model=model, r=r, n=n, dt=0.01, R=np.full(r, float(R)), n_scales=N, **kw)


def test_ito_correction_makes_the_update_unbiased():
    """Remark 3.1: for dy ~ N(0, dt I), E[exp(h.dy - dt/2 |h|^2)] = 1; without the
    -dt/2 |h|^2 term the mean would be exp(dt |h|^2 / 2)."""
    p = _problem(r=2, n=3)
    x = np.array([[0.9, -1.1], [0.3, 0.2], [1.3, 0.5]])
    rng = np.random.default_rng(5)
    M = 400_000
    dys = rng.normal(scale=math.sqrt(p.dt), size=(M, 2))
    for i in range(3):
        vals = np.exp(np.array([F.log_likelihood(p, x[i:i + 1], dy)[0] for dy in dys[:2000]]))
        # vectorised form of the same function on all draws
        h = x[i] ** 3
        ll = dys @ h - 0.5 * p.dt * np.sum(h * h)
        assert np.allclose(vals, np.exp(ll[:2000]), rtol=1e-13)
        w = np.exp(ll)
        se = w.std() / math.sqrt(M)
        assert abs(w.mean() - 1.0) < 4 * se
        assert abs(w.mean() - math.exp(0.5 * p.dt * np.sum(h * h))) > 4 * se or np.sum(h * h) < 1e-3


def test_log_likelihood_hand_values():
    p = _problem(r=2, n=2)
    x = np.array([[1.0, 2.0]])
    dy = np.array([0.1, -0.2])
    # h = (1, 8): h.dy = 0.1 - 1.6 = -1.5 ; dt/2 |h|^2 = 0.005 * 65 = 0.325
    assert F.log_likelihood(p, x, dy)[0] == pytest.approx(-1.825, abs=1e-14)
    pl = _problem(model="linear", r=2, n=2)
    assert F.log_likelihood(pl, x, dy)[0] == pytest.approx(0.1 - 0.4 - 0.005 * 5, abs=1e-14)


def test_signed_combination_against_linear_domain():
    """sum_j c_j e^{L_j} + c_{N+1} e^{ell}, evaluated directly in the linear domain."""
    rng = np.random.default_rng(1)
    for N in (1, 2, 3, 4):
        p = _problem(N=N, n=200)
        Lj = rng.normal(scale=0.3, size=(200, N))
        lw = rng.normal(scale=0.3, size=200)
        mask = np.zeros(200, bool)
        mask[7] = True
        out, clamps = F.combine(p, Lj, lw, mask)
        c = p.coef
        lin = np.exp(Lj) @ c[:N] + c[N] * np.exp(lw)
        mag = np.exp(Lj) @ np.abs(c[:N]) + abs(c[N]) * np.exp(lw)
        ok = (lin > 0) & ~mask
        # the linear-domain sum itself carries a rounding error ~ eps * mag / lin
        tol = 1e-13 * mag[ok] / lin[ok]
        assert np.all(np.abs(out[ok] - np.log(lin[ok])) <= tol)
        assert np.all(np.isneginf(out[~ok]))
        assert clamps == int(np.sum((lin <= 0) & ~mask))


def test_normalise_and_estimate_invariants():
    rng = np.random.default_rng(2)
    n, r = 500, 4
    x = rng.normal(size=(n, r))
    lw = rng.normal(scale=5.0, size=n)
    lam, h = F.normalise(lw)
    assert abs(np.sum(np.exp(h)) - 1.0) <= n * 2.0 ** -52
    mean, var, ess = F.estimate(x, h)
    assert 1.0 <= ess <= n
    # shift invariance
    lam2, h2 = F.normalise(lw + 1234.5)
    assert lam2 == pytest.approx(lam + 1234.5, abs=1e-9)
    m2, v2, e2 = F.estimate(x, h2)
    assert np.allclose(m2, mean, atol=1e-12) and np.allclose(v2, var, atol=1e-12)
    assert e2 == pytest.approx(ess, rel=1e-10)
    # equal weights -> ESS = n, mean/var are the plain sample moments
    m3, v3, e3 = F.estimate(x, F.normalise(np.zeros(n))[1])
    assert e3 == pytest.approx(n, rel=1e-12)
    assert np.allclose(m3, x.mean(0), atol=1e-12) and np.allclose(v3, x.var(0), atol=1e-12)
    # one finite weight -> ESS = 1 and the estimate is that node
    lw4 = np.full(n, -np.inf)
    lw4[17] = 3.0
    m4, v4, e4 = F.estimate(x, F.normalise(lw4)[1])
    assert e4 == 1.0 and np.array_equal(m4, x[17]) and np.all(v4 == 0)


def test_hand_computed_estimate():
    x = np.array([[0.0, 1.0], [2.0, 3.0]])
    h = np.log(np.array([0.25, 0.75]))
    mean, var, ess = F.estimate(x, h)
    assert np.allclose(mean, [1.5, 2.5])
    assert np.allclose(var, [0.75, 0.75])        # 0.25*2.25 + 0.75*0.25
    assert ess == pytest.approx(1.0 / (0.0625 + 0.5625))


def test_restart_rules():
    p = _problem(n=100, restart_interval=2, ess_frac=0.5)
    assert F.restart_due(p, 49.9, 1) and not F.restart_due(p, 50.0, 1)
    assert F.restart_due(p, 80.0, 4) and not F.restart_due(p, 80.0, 3)
    p1 = _problem(n=100, restart_interval=1, ess_frac=0.0)
    assert not F.restart_due(p1, 1.0, 2)   # iota = 1: no restart (restart remark)


def test_restart_translates_reference_nodes_and_uniform_init():
    p = _problem(model="cubic", r=3, n=64, R=0.5, N=2, restart_interval=2, ess_frac=0.0,
                 restart_init="uniform")
    u = sobol.nodes(sobol_poly_params(3, 1), sobol_scramble_params(3, 1), 64, 0.5)[1]
    st = F.init_state(p, u, np.zeros(3))
    tr = simulate("cubic", 3, 2, 0.01, seed=3)
    rec1, st = F.step(p, st, tr.dy[0])
    rec2, st2 = F.step(p, st, tr.dy[1])
    assert rec2.restarted and not rec1.restarted
    assert np.array_equal(st2.centre, rec2.mean)
    assert st2.u is st.u
    x_new = F.prepare(p, st2.u, st2.centre).x
    assert np.array_equal(x_new, st2.centre[None, :] + u.astype(np.float64))
    _, _, ess = F.estimate(x_new, st2.logw)
    assert ess == pytest.approx(64.0, rel=1e-12)
    assert st2.lognorm == rec2.lognorm


def test_kalman_steady_state_matches_riccati():
    """dP/dt = 2aP + 1 - P^2 has P_inf = a + sqrt(a^2 + 1); the Euler-discretised
    filter approaches it as dt -> 0."""
    a = -0.5
    rng = np.random.default_rng(0)
    dys = rng.normal(scale=0.01, size=(20000, 1))
    _, P = kalman.kalman_filter(dys, a, 0.001)
    assert P[-1, 0] == pytest.approx(a + math.sqrt(a * a + 1), rel=2e-3)


@pytest.mark.slow
def test_whole_filter_matches_kalman_on_linear_gaussian():
    """Linear-Gaussian model, first-order kernel, global box, no restart: the kernel
    propagation of a Gaussian is exactly Gaussian (closed form in test_oracle_kernel),
    so the filter mean must follow the exact discrete Kalman filter up to the quadrature
    error, which shrinks when n grows."""
    r, K, dt = 1, 100, 0.01
    tr = simulate("linear", r, K, dt, seed=11)
    km, kv = kalman.kalman_filter(tr.dy, -0.5, dt)
    errs = []
    for n in (1024, 4096):
        p = F.Problem(model="linear", r=r, n=n, dt=dt, R=np.full(r, 6.0), n_scales=1)
        u = sobol.nodes(sobol_poly_params(r, 1), sobol_scramble_params(r, 1), n, 6.0)[1]
        recs = F.run(p, F.init_state(p, u, np.zeros(r)), tr.dy)
        est = np.array([q.mean for q in recs])
        errs.append(float(np.sqrt(np.mean((est - km) ** 2))))
    p_inf = math.sqrt(1.25) - 0.5
    assert errs[1] < 0.005 * math.sqrt(p_inf)
    assert errs[1] < errs[0]


def test_metrics_hand_values():
    truth = np.array([[0.0, 0.0], [1.0, 1.0]])
    est = np.array([[1.0, 1.0], [1.0, 3.0]])
    # squared errors per step: 2, 4 ; RMSE = sqrt(6 / 4) ; ME = (sqrt(1) + sqrt(2)) / 2
    assert metrics.rmse(est, truth) == pytest.approx(math.sqrt(1.5))
    assert metrics.me(est, truth) == pytest.approx((1.0 + math.sqrt(2.0)) / 2)
