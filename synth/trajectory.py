"""Euler--Maruyama truth and observation increments for the filtering problem.

The problem ("Continuous-Time Nonlinear Filtering Problem", eq. NonlinearFilter) is
dX = f(X)dt + dV, dY = h(X)dt + dW with unit-covariance Brownian motions.  The experiments
discretise both SDEs with Euler--Maruyama at the filter step dt ("Large-Scale Scalability
Test", setup).  The observation of step k uses the state after the step:

    x_k  = x_{k-1} + f(x_{k-1}) dt + sqrt(dt) xi_k,
    dy_k = h(x_k) dt + sqrt(dt) eta_k,            xi_k, eta_k ~ N(0, I).

Models (m = r, componentwise sensors):
    "cubic"    : f(x) = cos(x),   h(x) = x^3
    "linear"   : f(x) = a x,      h(x) = x      (a = model_a, -0.5 by default)
    "paper_e1" : f(x) = sin(x) (A x) + sin(2x) (A1 x) elementwise, A / A1 upper bidiagonal with
                 diagonal -0.5 / -0.3 and superdiagonal 0.1 / 0.3; h(x) = (x - 100)^3 (the
                 large-scale scalability test of the paper's numerical section)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Trajectory:
    x0: np.ndarray      # [r]    initial state
    x: np.ndarray       # [K][r] true states x_1..x_K
    dy: np.ndarray      # [K][r] observation increments dy_1..dy_K


def _drift(model: str, a: float, x: np.ndarray) -> np.ndarray:
    if model == "cubic":
        return np.cos(x)
    if model == "linear":
        return a * x
    if model == "paper_e1":   # sin(x) (A x) + sin(2x) (A1 x), A, A1 upper bidiagonal
        ax = -0.5 * x
        ax[:-1] += 0.1 * x[1:]
        a1x = -0.3 * x
        a1x[:-1] += 0.3 * x[1:]
        return np.sin(x) * ax + np.sin(2 * x) * a1x
    raise ValueError(model)


def _sensor(model: str, x: np.ndarray) -> np.ndarray:
    if model == "cubic":
        return x ** 3
    if model == "linear":
        return x.copy()
    if model == "paper_e1":
        return (x - 100.0) ** 3
    raise ValueError(model)


def _noise_u(noise, x):
    U = noise["u"] * (1.0 + noise["u_kappa"] * np.sin(x) ** 2)
    U[:noise.get("u_zero", 0)] = 0.0
    return U


def _noise_v(noise, x):
    return noise["v"] * (1.0 + noise["v_kappa"] * np.sin(x) ** 2)


def simulate(model: str, r: int, steps: int, dt: float, seed: int,
             model_a: float = -0.5, prior_mean: float = 0.0, prior_std: float = 1.0,
             noise: dict | None = None) -> Trajectory:
    """Seeded Euler--Maruyama run; x_0 ~ N(prior_mean, prior_std^2 I).  noise: diagonal
    noise coefficients U_d(x) = u (1 + u_kappa sin^2 x_d) (zero for the first u_zero
    coordinates) and V_d(x) = v (1 + v_kappa sin^2 x_d); None: unit noise."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(seed) ^ np.uint64(0x7A11EC7)))
    x = prior_mean + prior_std * rng.standard_normal(r)
    x0 = x.copy()
    xs = np.empty((steps, r))
    dys = np.empty((steps, r))
    sq = np.sqrt(dt)
    for k in range(steps):
        su = 1.0 if noise is None else _noise_u(noise, x)
        x = x + _drift(model, model_a, x) * dt + su * sq * rng.standard_normal(r)
        xs[k] = x
        sv = 1.0 if noise is None else _noise_v(noise, x)
        dys[k] = _sensor(model, x) * dt + sv * sq * rng.standard_normal(r)
    return Trajectory(x0=x0, x=xs, dy=dys)
