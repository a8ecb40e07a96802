"""Drift f, divergence div f and sensor h of the workload models, in float64.

cubic    : f(x) = cos(x) componentwise, div f = -sum_d sin(x_d), h(x) = x^3
linear   : f(x) = a x,                  div f = a r,              h(x) = x
paper_e1 : the large-scale scalability test of "Large-Scale Scalability Test":
           f(x) = sin(x) * (A x) + sin(2x) * (A1 x) elementwise, A and A1 upper bidiagonal
           with diagonal -0.5 / -0.3 and superdiagonal 0.1 / 0.3, h(x) = (x - 100)^3;
           div f = sum_d [cos(x_d) (A x)_d - 0.5 sin(x_d) + 2 cos(2 x_d) (A1 x)_d - 0.3 sin(2 x_d)]

``complex_step_divergence`` is the complex-step formula of "Numerical Divergence Calculation"
(the boxed formula there):
div f(x) ~= sum_k Im f_k(x + i h e_k) / h, used to cross-check the closed forms.
"""
from __future__ import annotations

import numpy as np


def _bidiag(x: np.ndarray, diag: float, sup: float) -> np.ndarray:
    """(B x) for the upper-bidiagonal B with constant diagonal and superdiagonal."""
    out = diag * x
    out[..., :-1] += sup * x[..., 1:]
    return out


def drift(model: str, x: np.ndarray, a: float = -0.5) -> np.ndarray:
    if model == "cubic":
        return np.cos(x)
    if model == "linear":
        return a * x
    if model == "paper_e1":
        return np.sin(x) * _bidiag(x, -0.5, 0.1) + np.sin(2 * x) * _bidiag(x, -0.3, 0.3)
    raise ValueError(model)


def divergence(model: str, x: np.ndarray, a: float = -0.5) -> np.ndarray:
    if model == "cubic":
        return -np.sin(x).sum(axis=-1)
    if model == "linear":
        return np.full(x.shape[:-1], a * x.shape[-1])
    if model == "paper_e1":
        return (np.cos(x) * _bidiag(x, -0.5, 0.1) - 0.5 * np.sin(x)
                + 2 * np.cos(2 * x) * _bidiag(x, -0.3, 0.3) - 0.3 * np.sin(2 * x)).sum(axis=-1)
    raise ValueError(model)


def sensor(model: str, x: np.ndarray) -> np.ndarray:
    if model == "cubic":
        return x ** 3
    if model == "linear":
        return x.copy()
    if model == "paper_e1":
        return (x - 100.0) ** 3
    raise ValueError(model)


def complex_step_divergence(model: str, x: np.ndarray, a: float = -0.5,
                            h: float = 1e-20) -> np.ndarray:
    """Sum over k of Im f_k(x + i h e_k) / h for each row of x."""
    x = np.atleast_2d(x).astype(np.complex128)
    out = np.zeros(x.shape[0])
    for k in range(x.shape[1]):
        xp = x.copy()
        xp[:, k] += 1j * h
        out += np.imag(drift(model, xp, a)[:, k]) / h
    return out


# ---- diagonal noise coefficients (Section "General Nonlinear Filtering with Noise
# Coefficients"): dX = f dt + U(X) dV, dY = h dt + V(X) dW with
#     U_d(x) = u (1 + u_kappa sin^2 x_d), zero for the first u_zero coordinates (a singular),
#     V_d(x) = v (1 + v_kappa sin^2 x_d),
# a = U U^T = diag(U_d^2), b = V V^T = diag(V_d^2).

def state_noise(noise: dict, x: np.ndarray) -> np.ndarray:
    U = noise["u"] * (1.0 + noise["u_kappa"] * np.sin(x) ** 2)
    U[..., :noise.get("u_zero", 0)] = 0.0
    return U


def obs_noise(noise: dict, x: np.ndarray) -> np.ndarray:
    return noise["v"] * (1.0 + noise["v_kappa"] * np.sin(x) ** 2)


def kernel_metric(noise: dict, x: np.ndarray):
    """(a(x)^+ as the diagonal [..][r], 1/2 log det_+ a(x) [..]): the pseudo-inverse and
    the determinant over the positive entries."""
    a = state_noise(noise, x) ** 2
    pos = a > 0.0
    minv = np.where(pos, 1.0 / np.where(pos, a, 1.0), 0.0)
    hld = 0.5 * np.sum(np.where(pos, np.log(np.where(pos, a, 1.0)), 0.0), axis=-1)
    return minv, hld
