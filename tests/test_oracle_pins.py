"""Pins for the oracle functions that the restart, the initial state and the network's
training rest on: the Gaussian restart weights, the prior weights, Adam beyond its first
step and the network's input features.  Each is checked against an independent library
routine (scipy's normal densities, torch's Adam) and against values worked out by hand,
so that a dropped term, a wrong floor or a variance used as a standard deviation fails."""
import math

import numpy as np
import pytest

from oracle import filter as F, mlp


def _problem(r=2, n=4, R=0.4, **kw):
    return F.Problem(model="cubic", r=r, n=n, dt=0.01, R=np.full(r, float(R)), n_scales=2, **kw)


# ---- restart weights, Gaussian branch (reading A6: N(c, diag(max(v, (R/4)^2)))) --------

def test_restart_logw_two_points_closed_form():
    """Two nodes in 1-D: the normalised weight of node 1 is the logistic function of the
    difference of the two Gaussian exponents, with the variance floored at (R/4)^2."""
    R = 0.4
    p = _problem(r=1, n=2, R=R)
    x = np.array([[0.10], [0.25]])
    c = np.array([0.05])
    for var, v_used in ((0.001, 0.01), (0.04, 0.04)):   # below and above the floor (R/4)^2 = 0.01
        lw = F.restart_logw(p, x, c, np.array([var]))
        d1, d2 = 0.05 ** 2, 0.20 ** 2
        w1 = 1.0 / (1.0 + math.exp(-(d2 - d1) / (2.0 * v_used)))
        assert lw[0] == pytest.approx(math.log(w1), abs=1e-13)
        assert lw[1] == pytest.approx(math.log(1.0 - w1), abs=1e-13)
    # hand values: v = 0.01: exponent gap (0.04 - 0.0025) / 0.02 = 1.875
    lw = F.restart_logw(p, x, c, np.array([0.0]))
    assert lw[0] == pytest.approx(-math.log1p(math.exp(-1.875)), abs=1e-13)
    assert lw[1] == pytest.approx(-1.875 - math.log1p(math.exp(-1.875)), abs=1e-13)


def test_restart_logw_against_scipy_normal_densities():
    """Several dimensions, mixed sides of the floor, per-dimension half-widths: the
    normalised log-density of independent normals from scipy."""
    from scipy.special import logsumexp
    from scipy.stats import norm
    rng = np.random.default_rng(3)
    r, n = 3, 50
    half = np.array([0.3, 0.8, 0.5])
    p = _problem(r=r, n=n, R=0.3)
    c = np.array([0.2, -1.0, 0.4])
    x = c + rng.uniform(-1, 1, size=(n, r)) * half
    var = np.array([0.001, 0.5, (0.5 / 4) ** 2 * 0.999])
    lw = F.restart_logw(p, x, c, var, half)
    sd = np.sqrt(np.maximum(var, (half / 4) ** 2))
    ref = norm.logpdf(x, loc=c, scale=sd).sum(axis=1)
    ref -= logsumexp(ref)
    assert np.max(np.abs(lw - ref)) < 1e-12
    assert abs(logsumexp(lw)) < 1e-13
    # the problem's own R is used when no half-widths are given
    lw_r = F.restart_logw(p, x, c, var)
    sd_r = np.sqrt(np.maximum(var, (0.3 / 4) ** 2))
    ref_r = norm.logpdf(x, loc=c, scale=sd_r).sum(axis=1)
    assert np.max(np.abs(lw_r - (ref_r - logsumexp(ref_r)))) < 1e-12


def test_restart_logw_uniform_branch():
    p = _problem(r=2, n=8, restart_init="uniform")
    lw = F.restart_logw(p, np.zeros((8, 2)), np.zeros(2), np.ones(2))
    assert np.all(lw == -math.log(8))


# ---- prior weights: log sigma_0 for x_0 ~ N(mu0, s0^2 I) ---------------------------------

def test_prior_logw_hand_values():
    p = _problem(r=3, prior_mean=0.5, prior_var=4.0)
    x = np.array([[0.5, 0.5, 0.5], [2.5, 0.5, -1.5]])
    lw = F.prior_logw(p, x)
    const = -1.5 * math.log(2 * math.pi * 4.0)
    assert lw[0] == pytest.approx(const, abs=1e-13)                    # at the mean
    assert lw[1] == pytest.approx(const - (4.0 + 4.0) / 8.0, abs=1e-13)  # |x - mu|^2 = 8, 2 s0^2 = 8


def test_prior_logw_against_scipy():
    from scipy.stats import multivariate_normal
    rng = np.random.default_rng(4)
    for mu, var in ((0.0, 1.0), (-0.3, 0.25), (1.2, 2.5)):
        p = _problem(r=4, prior_mean=mu, prior_var=var)
        x = rng.normal(size=(20, 4))
        ref = multivariate_normal(mean=np.full(4, mu), cov=var * np.eye(4)).logpdf(x)
        assert np.max(np.abs(F.prior_logw(p, x) - ref)) < 1e-12


# ---- Adam (Kingma & Ba 2015) beyond the first step ---------------------------------------

def test_adam_two_steps_by_hand():
    """t = 1: m = 0.05, v = 2.5e-4 -> step lr; t = 2 with g = -0.25: m = 0.02,
    v = 0.999 * 2.5e-4 + 0.001 * 0.0625 = 3.1225e-4, bias-corrected 0.02 / 0.19 and
    3.1225e-4 / 0.001999, so p = 0.9 - 0.1 * 0.1052632 / 0.3952253 = 0.8733665."""
    p = {"w": np.array([1.0])}
    m = {"w": np.zeros(1)}
    v = {"w": np.zeros(1)}
    mlp.adam_step(p, {"w": np.array([0.5])}, m, v, 1, lr=0.1)
    assert p["w"][0] == pytest.approx(0.9, abs=1e-7)
    mlp.adam_step(p, {"w": np.array([-0.25])}, m, v, 2, lr=0.1)
    assert m["w"][0] == pytest.approx(0.02, abs=1e-15)
    assert v["w"][0] == pytest.approx(3.1225e-4, abs=1e-15)
    assert p["w"][0] == pytest.approx(0.8733665, abs=1e-6)


def test_adam_matches_torch_optimizer_over_many_steps():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    w0 = rng.normal(size=(3, 4))
    grads = [rng.normal(size=(3, 4)) * (0.1 + k) for k in range(12)]
    p = {"w": w0.copy()}
    m = {"w": np.zeros_like(w0)}
    v = {"w": np.zeros_like(w0)}
    tw = torch.tensor(w0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tw], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    for t, g in enumerate(grads, start=1):
        mlp.adam_step(p, {"w": g}, m, v, t, lr=3e-3)
        opt.zero_grad()
        tw.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    assert np.max(np.abs(p["w"] - tw.detach().numpy())) < 1e-12


# ---- network input features ----------------------------------------------------------

def test_features_hand_values():
    z = mlp.features(np.array([1.0, -2.0]), np.array([4.0, -1e-18]), np.array([0.1, -0.2]), 0.01,
                     np.array([0.25, -2.5]))
    # [x_hat - c; sqrt(max(v, 0)); dy / sqrt(dt)]
    assert np.allclose(z, [0.75, 0.5, 2.0, 0.0, 1.0, -2.0], rtol=0, atol=1e-15)
