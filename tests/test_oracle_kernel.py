"""Pins for the oracle's kernel sums ("Solving Kolmogorov Equations via Low-Discrepancy
Sampling and Kernel Approximation", "Log-Domain Computation" prediction)."""
import math

import numpy as np
import pytest

from oracle import filter as F, model as mdl, sobol
from synth import sobol_poly_params, sobol_scramble_params


def _problem(model, r, n, R, N=1, dt=0.01, a=-0.5):
    return F.Problem(model=model, r=r, n=n, dt=dt, R=np.full(r, float(R)), n_scales=N, model_a=a)


def _nodes(r, n, R, seed=1):
    return sobol.nodes(sobol_poly_params(r, seed), sobol_scramble_params(r, seed), n, R)[1]


@pytest.mark.parametrize("r", [1, 2, 3])
def test_brute_force_linear_domain(r):
    """Naive linear-domain double sum with the kernel written in completed-square form
    c_tau exp(-|y - (x - tau f(x))|^2 / (2 tau) - tau div f(x)), an algebraically
    equivalent route to eq. kernel; no log-sum-exp, no max shift."""
    n, R = 48, 0.6
    p = _problem("cubic", r, n, R, N=3, dt=0.05)
    u = _nodes(r, n, R)
    prep = F.prepare(p, u, np.full(r, 0.4))
    rng = np.random.default_rng(r)
    logw = rng.normal(size=n)
    prep.mask[5] = True          # a boundary node: excluded as a source
    L = F.kernel_lse(p, prep, logw)
    wq = np.prod(2 * p.R) / n
    for i in range(n):
        for j, tau in enumerate(p.taus):
            xt = prep.x[i] - tau * prep.f[i]
            acc = 0.0
            for s in range(n):
                if prep.mask[s]:
                    continue
                d2 = float(np.sum((prep.x[s] - xt) ** 2))
                k = (2 * math.pi * tau) ** (-r / 2) * math.exp(-d2 / (2 * tau) - tau * prep.divf[i])
                acc += k * wq * math.exp(logw[s])
            assert L[i, j] == pytest.approx(math.log(acc), abs=1e-12, rel=1e-12)


@pytest.mark.parametrize("r,n,R,dt,tol", [(1, 1 << 14, 6.0, 0.01, 2e-4), (2, 1 << 14, 2.0, 0.08, 4e-3)])
def test_linear_drift_gaussian_closed_form(r, n, R, dt, tol):
    """f(x) = a x and weights N(m, P I):  int K_tau(x, y) N(y; m, P) dy
    = e^{-a tau r} N(x (1 - a tau); m, (P + tau) I), because the kernel is a Gaussian in y
    centred at x - tau f(x) times e^{-tau div f}.  Dense QMC nodes approximate the integral."""
    a, m, P = -0.5, 0.3, 0.4
    p = _problem("linear", r, n, R, N=2, dt=dt, a=a)
    u = _nodes(r, n, R, seed=2)
    prep = F.prepare(p, u, np.zeros(r))
    d = prep.x - m
    logw = -0.5 * np.sum(d * d, axis=1) / P - 0.5 * r * math.log(2 * math.pi * P)
    inner = np.where(np.all(np.abs(prep.x - m) < 1.2, axis=1))[0][:40]
    for i in inner:
        L = F.kernel_lse(p, prep, logw, t0=int(i), t1=int(i) + 1)[0]
        for j, tau in enumerate(p.taus):
            xt = prep.x[i] * (1 - a * tau)
            v = P + tau
            ref = -a * tau * r - 0.5 * np.sum((xt - m) ** 2) / v - 0.5 * r * math.log(2 * math.pi * v)
            assert L[j] == pytest.approx(ref, abs=tol)


def test_zero_drift_kernel_integrates_to_one():
    """f = 0: sum_s K(x_i, x_s) w_q ~ int K dy = 1 (the first-order kernel theorem)
    away from the faces."""
    p = _problem("linear", 1, 4096, 2.0, N=1, dt=0.01, a=0.0)
    u = _nodes(1, 4096, 2.0, seed=3)
    prep = F.prepare(p, u, np.zeros(1))
    L = F.kernel_lse(p, prep, np.zeros(4096))[:, 0]
    inner = np.abs(prep.x[:, 0]) < 1.5
    assert np.max(np.abs(L[inner])) < 1e-4


def test_drift_is_evaluated_at_the_target():
    """Remark after eq. L_Delta_t: the first argument x is the evaluation point.  With
    one source, L(i) depends on f(x_i) only, not on f(x_s)."""
    p = _problem("cubic", 1, 2, 1.0, N=1, dt=0.1)
    u = np.array([[0.1], [0.5]], dtype=np.float32)
    prep = F.prepare(p, u, np.zeros(1))
    lw = np.array([0.0, -np.inf])  # only source 0 contributes
    L1 = F.kernel_lse(p, prep, lw)[:, 0]
    prep.f[0] += 1.0              # change the drift at the source/target 0
    L2 = F.kernel_lse(p, prep, lw)[:, 0]
    assert L1[1] == L2[1]        # target 1 unchanged: f of the source is not used
    assert L1[0] != L2[0]


def test_masked_target_is_minus_inf_and_masked_source_excluded():
    p = _problem("cubic", 2, 16, 0.5, N=2, dt=0.02)
    u = _nodes(2, 16, 0.5)
    prep = F.prepare(p, u, np.zeros(2))
    lw = np.zeros(16)
    base, _ = F.predict(p, prep, lw)
    prep.mask[3] = True
    masked, _ = F.predict(p, prep, lw)
    assert masked[3] == -np.inf
    lw2 = lw.copy()
    lw2[3] = -np.inf
    prep.mask[3] = False
    excl, _ = F.predict(p, prep, lw2)
    keep = np.arange(16) != 3
    assert np.allclose(masked[keep], excl[keep], rtol=0, atol=1e-12)


def test_boundary_mask_rule():
    """Nodes within omega = 1e-12 R of a face are on the boundary ("Algorithm for Kolmogorov
    Equation", step 3)."""
    R = np.array([0.3, 0.3])
    u = np.array([[0.3, 0.0], [0.0, -0.3], [0.2999, 0.1], [np.float32(0.3) * (1 - 2 ** -23), 0.0]],
                 dtype=np.float32)
    m = F.boundary_mask(u, R)
    assert m.tolist() == [True, True, False, False]


@pytest.mark.parametrize("model", ["cubic", "linear", "paper_e1"])
def test_divergence_closed_form_vs_complex_step(model):
    """Complex-step divergence ("Numerical Divergence Calculation"): sum_k Im f_k(x + i h e_k) / h, h = 1e-20, against
    the closed forms."""
    rng = np.random.default_rng(0)
    x = rng.normal(size=(20, 7))
    cs = mdl.complex_step_divergence(model, x, a=-0.5)
    cf = mdl.divergence(model, x, a=-0.5)
    assert np.allclose(cs, cf, rtol=1e-14, atol=1e-14)


def test_paper_e1_model_hand_values_and_matrix_form():
    """The large-scale test's drift with its matrices written out (upper bidiagonal: the
    superdiagonal couples x_d to x_{d+1}); sensor (x - 100)^3."""
    x = np.array([[1.0, 2.0]])
    # A x = (-0.5 + 0.2, -1.0), A1 x = (-0.3 + 0.6, -0.6)
    f = mdl.drift("paper_e1", x)
    assert f[0, 0] == pytest.approx(np.sin(1.0) * -0.3 + np.sin(2.0) * 0.3, abs=1e-15)
    assert f[0, 1] == pytest.approx(np.sin(2.0) * -1.0 + np.sin(4.0) * -0.6, abs=1e-15)
    rng = np.random.default_rng(3)
    r = 9
    A = np.diag(np.full(r, -0.5)) + np.diag(np.full(r - 1, 0.1), k=1)
    A1 = np.diag(np.full(r, -0.3)) + np.diag(np.full(r - 1, 0.3), k=1)
    xs = rng.normal(size=(5, r))
    ref = np.sin(xs) * (xs @ A.T) + np.sin(2 * xs) * (xs @ A1.T)
    assert np.allclose(mdl.drift("paper_e1", xs), ref, rtol=0, atol=1e-14)
    assert mdl.sensor("paper_e1", np.array([[0.0, 101.0]])).tolist() == [[-1e6, 1.0]]
