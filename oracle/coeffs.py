"""Coefficients of the N-scale kernel ("High-Order Kernel Construction", eq. general_kernel).

Scales s_j = 2^(j-1), j = 1..N, and eliminated error orders mu_k = 3/2, 2, 5/2, ...
(the example given after the expansion of L_{dt/s_j}).  The N+1 constraints are
constant-term matching, dt-term matching and elimination of the N-1 error orders,
V c = d with the generalised Vandermonde matrix V, solved by Cramer's rule as the
paper states.  c[N] is the coefficient of the identity (Dirac) term.
"""
from __future__ import annotations

import numpy as np


def scales(n_scales: int) -> np.ndarray:
    return np.array([2.0 ** j for j in range(n_scales)])


def error_orders(n_scales: int) -> np.ndarray:
    return np.array([1.5 + 0.5 * k for k in range(n_scales - 1)])


def vandermonde(n_scales: int) -> tuple[np.ndarray, np.ndarray]:
    s = scales(n_scales)
    mu = error_orders(n_scales)
    N = n_scales
    V = np.zeros((N + 1, N + 1))
    d = np.zeros(N + 1)
    V[0, :] = 1.0
    d[0] = 1.0
    V[1, :N] = 1.0 / s
    d[1] = 1.0
    for k in range(N - 1):
        V[2 + k, :N] = s ** (-mu[k])
    return V, d


def kernel_coefficients(n_scales: int) -> np.ndarray:
    """c_1..c_{N+1} by Cramer's rule c_j = det V_j / det V."""
    if not 1 <= n_scales <= 6:
        raise ValueError("n_scales must be in 1..6")
    V, d = vandermonde(n_scales)
    det = np.linalg.det(V)
    c = np.empty(n_scales + 1)
    for j in range(n_scales + 1):
        Vj = V.copy()
        Vj[:, j] = d
        c[j] = np.linalg.det(Vj) / det
    return c
