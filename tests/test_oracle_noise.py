"""Pins for the oracle's diagonal noise coefficients (the section on filtering with noise
coefficients, table of invertible and singular formulas): unit coefficients reproduce the
unit-noise filter exactly; a constant coefficient sigma turns the linear-drift Gaussian
closed form into N(x(1 - a tau); m, P + tau sigma^2); with zero drift and state-dependent
a(x) evaluated at the target the kernel still integrates to one; a singular coordinate
(the pseudo-inverse) drops out of the distance, so its integral is the box width times
the prefactor's (2 pi tau)^(-1/2); the
b^-1-weighted update is unbiased under dy ~ N(0, b dt); and hand values of the metric."""
import math

import numpy as np
import pytest

from oracle import filter as F, model as mdl, sobol
from synth import simulate, sobol_poly_params, sobol_scramble_params


def _nodes(r, n, R, seed=1):
    return sobol.nodes(sobol_poly_params(r, seed), sobol_scramble_params(r, seed), n, R)[1]


def _prob(model, r, n, R, N=1, noise=None, a=-0.5):
    return F.Problem(model=model, r=r, n=n, dt=0.01, R=np.full(r, R), n_scales=N, noise=noise, model_a=a)


def test_unit_coefficients_reproduce_unit_noise():
    r, n, R = 3, 512, 0.6
    u = _nodes(r, n, R)
    unit = dict(u=1.0, u_kappa=0.0, u_zero=0, v=1.0, v_kappa=0.0)
    p0, p1 = _prob("cubic", r, n, R, 2), _prob("cubic", r, n, R, 2, noise=unit)
    c = np.array([0.1, -0.2, 0.3])
    st = F.init_state(p0, u, c)
    L0 = F.kernel_lse(p0, F.prepare(p0, u, c), st.logw)
    L1 = F.kernel_lse(p1, F.prepare(p1, u, c), st.logw)
    assert np.max(np.abs(L0 - L1)) <= 1e-12
    x = F.prepare(p0, u, c).x
    dy = np.array([0.02, -0.01, 0.05])
    assert np.max(np.abs(F.log_likelihood(p0, x, dy) - F.log_likelihood(p1, x, dy))) <= 1e-12


def test_constant_coefficient_linear_gaussian_closed_form():
    """f = a x, phi = N(m, P): int K(x, y) phi(y) dy = e^{-a tau} N(x (1 - a tau); m, P + tau sigma^2)."""
    r, n, R, a, tau, sig = 1, 1 << 14, 6.0, -0.5, 0.01, 1.7
    u = _nodes(r, n, R)
    p = _prob("linear", r, n, R, noise=dict(u=sig, u_kappa=0.0, u_zero=0, v=1.0, v_kappa=0.0), a=a)
    prep = F.prepare(p, u, np.zeros(r))
    m, P = 0.4, 0.3
    lw = -0.5 * (prep.x[:, 0] - m) ** 2 / P - 0.5 * math.log(2 * math.pi * P)
    L = F.kernel_lse(p, prep, lw)[:, 0]
    xt = prep.x[:, 0] * (1 - a * tau)
    S = P + tau * sig ** 2
    ref = -a * tau - 0.5 * (xt - m) ** 2 / S - 0.5 * math.log(2 * math.pi * S)
    sel = np.abs(prep.x[:, 0]) < 2.5
    assert np.max(np.abs(np.exp(L[sel]) - np.exp(ref[sel]))) <= 2e-4 * np.max(np.exp(ref))


def test_state_dependent_coefficient_kernel_integrates_to_one():
    r, n, R = 2, 1 << 14, 3.0
    u = _nodes(r, n, R)
    p = _prob("linear", r, n, R, noise=dict(u=0.8, u_kappa=0.7, u_zero=0, v=1.0, v_kappa=0.0), a=0.0)
    prep = F.prepare(p, u, np.zeros(r))
    L = F.kernel_lse(p, prep, np.zeros(n), 0, 200)[:, 0]
    inner = np.all(np.abs(prep.x[:200]) < 2.0, axis=1)
    assert np.max(np.abs(np.exp(L[inner]) - 1.0)) <= 2e-2


def test_singular_coordinate_integrates_to_box_width():
    """The printed kernel keeps the prefactor (2 pi tau)^(-r/2) with the full r while the
    pseudo-inverse removes the singular coordinate from the exponent, so integrating over
    the box gives 2R (2 pi tau)^(-1/2) for one singular coordinate."""
    r, n, R = 2, 1 << 14, 2.0
    u = _nodes(r, n, R)
    p = _prob("linear", r, n, R, noise=dict(u=0.5, u_kappa=0.0, u_zero=1, v=1.0, v_kappa=0.0), a=0.0)
    prep = F.prepare(p, u, np.zeros(r))
    assert np.all(prep.minv[:, 0] == 0.0) and np.allclose(prep.minv[:, 1], 4.0)
    assert np.allclose(prep.hld, 0.5 * math.log(0.25))   # det_+ over the positive entry only
    L = F.kernel_lse(p, prep, np.zeros(n), 0, 200)[:, 0]
    inner = np.abs(prep.x[:200, 1]) < 1.2
    assert np.max(np.abs(np.exp(L[inner]) * math.sqrt(2 * math.pi * p.dt) / (2 * R) - 1.0)) <= 2e-2


def test_weighted_update_is_unbiased():
    noise = dict(u=1.0, u_kappa=0.0, u_zero=0, v=0.6, v_kappa=0.9)
    p = _prob("cubic", 2, 4, 1.0, noise=noise)
    x = np.array([[0.9, -1.1]])
    b = mdl.obs_noise(noise, x)[0] ** 2
    rng = np.random.default_rng(7)
    M = 400_000
    dys = rng.normal(size=(M, 2)) * np.sqrt(b * p.dt)
    h = x[0] ** 3
    ll = np.sum((h * dys - 0.5 * p.dt * h * h) / b, axis=1)
    assert np.allclose(F.log_likelihood(p, np.repeat(x, 5, axis=0), dys[0]), ll[0], rtol=1e-13)
    w = np.exp(ll)
    assert abs(w.mean() - 1.0) < 4 * w.std() / math.sqrt(M)


def test_metric_hand_values():
    noise = dict(u=0.5, u_kappa=1.0, u_zero=0, v=1.0, v_kappa=0.0)
    minv, hld = mdl.kernel_metric(noise, np.array([[math.pi / 2, 0.0]]))
    # U = 0.5 (1 + sin^2): 1.0 at pi/2, 0.5 at 0 -> a = 1, 0.25
    assert np.allclose(minv, [[1.0, 4.0]]) and np.allclose(hld, [0.5 * math.log(0.25)])


def test_simulation_with_noise_coefficients_is_seeded():
    noise = dict(u=0.5, u_kappa=0.5, u_zero=1, v=2.0, v_kappa=0.0)
    a = simulate("cubic", 3, 5, 0.01, seed=3, noise=noise)
    b = simulate("cubic", 3, 5, 0.01, seed=3, noise=noise)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.dy, b.dy)
    # the first coordinate has no state noise: it follows the drift alone
    x = a.x0[0]
    for k in range(5):
        x = x + math.cos(x) * 0.01
        assert a.x[k, 0] == pytest.approx(x, abs=1e-12)
