"""Drift f, divergence div f and sensor h of the two workload models, in float64.

cubic  : f(x) = cos(x) componentwise, div f = -sum_d sin(x_d), h(x) = x^3
linear : f(x) = a x,                  div f = a r,              h(x) = x

``complex_step_divergence`` is the complex-step formula of Section 6 (eq. boxed there):
div f(x) ~= sum_k Im f_k(x + i h e_k) / h, used to cross-check the closed forms.
"""
from __future__ import annotations

import numpy as np


def drift(model: str, x: np.ndarray, a: float = -0.5) -> np.ndarray:
    if model == "cubic":
        return np.cos(x)
    if model == "linear":
        return a * x
    raise ValueError(model)


def divergence(model: str, x: np.ndarray, a: float = -0.5) -> np.ndarray:
    if model == "cubic":
        return -np.sin(x).sum(axis=-1)
    if model == "linear":
        return np.full(x.shape[:-1], a * x.shape[-1])
    raise ValueError(model)


def sensor(model: str, x: np.ndarray) -> np.ndarray:
    if model == "cubic":
        return x ** 3
    if model == "linear":
        return x.copy()
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
