"""Exact discrete Kalman filter for the Euler-discretised linear-Gaussian model.

Model (componentwise, unit noise): x_k = (1 + a dt) x_{k-1} + sqrt(dt) xi_k,
dy_k = dt x_k + sqrt(dt) eta_k, x_0 ~ N(m0, P0).  The components are independent, so
the filter is r scalar filters.  This is the discrete counterpart of the Kalman--Bucy
filter the paper compares against in "Linear Filtering Benchmark".
"""
from __future__ import annotations

import numpy as np


def kalman_filter(dys: np.ndarray, a: float, dt: float, m0: float = 0.0, P0: float = 1.0):
    K, r = dys.shape
    m = np.full(r, m0, dtype=np.float64)
    P = np.full(r, P0, dtype=np.float64)
    means = np.empty((K, r))
    vars_ = np.empty((K, r))
    F = 1.0 + a * dt
    for k in range(K):
        m = F * m
        P = F * F * P + dt
        S = dt * dt * P + dt          # innovation variance of dy = dt x + sqrt(dt) eta
        G = P * dt / S
        m = m + G * (dys[k] - dt * m)
        P = (1.0 - G * dt) * P
        means[k] = m
        vars_[k] = P
    return means, vars_
