"""Halton and Faure node sets (Appendix A, "Halton Sequence" and "Faure Sequence"), the
paper's low-dimensional alternatives to Sobol nodes.

TEST INFRASTRUCTURE: only the tests, the smoke check and the bench's CPU-baseline leg may use
this module; it shares no code with the CUDA path.

Halton: coordinate d (1-based) of point k is the radical inverse of k in the d-th prime
p_d, phi_p(k) = sum_i k_i p^-(i+1) over the base-p digits k_i of k (least significant
first).  Faure: one base p, the smallest prime >= r; coordinate d of point k is
sum_i y_i p^-(i+1) with y = C^(d) k mod p, C^(d) = P^(d-1) mod p, P_ij = binom(j, i) (the
matrix power is taken here by repeated multiplication, as written in the appendix).

Exact arithmetic: with M digits and p^M <= 2^53 the value is the integer
R = sum_i y_i p^(M-1-i) over p^M, and R / p^M is evaluated by Python's correctly rounded
integer division, so the float64 value does not depend on M.  Box coordinates:
u = R_d (2 phi - 1) in float64 (three rounded operations), then rounded to float32.  The
sequences start at index `first` (1 by default: point 0 is the corner of the box).
"""
from __future__ import annotations

import numpy as np


def first_primes(count: int) -> list[int]:
    out, c = [], 2
    while len(out) < count:
        if all(c % q for q in out if q * q <= c):
            out.append(c)
        c += 1
    return out


def smallest_prime_at_least(m: int) -> int:
    c = max(2, m)
    while any(c % q == 0 for q in range(2, int(c ** 0.5) + 1)):
        c += 1
    return c


def max_digits(p: int) -> int:
    """Largest M with p^M <= 2^53."""
    M = 0
    while p ** (M + 1) <= 2 ** 53:
        M += 1
    return M


def digits(k: int, p: int, M: int) -> list[int]:
    out = []
    for _ in range(M):
        out.append(k % p)
        k //= p
    assert k == 0, "index needs more digits than the exact range allows"
    return out


def _value(y: list[int], p: int) -> float:
    M = len(y)
    R = 0
    for yi in y:            # y_0 is the most significant digit of the fraction
        R = R * p + yi
    return R / p ** M       # correctly rounded quotient of exact integers


def halton_unit(n: int, r: int, first: int = 1) -> np.ndarray:
    ps = first_primes(r)
    out = np.empty((n, r))
    for d, p in enumerate(ps):
        M = max_digits(p)
        for i in range(n):
            out[i, d] = _value(digits(first + i, p, M), p)
    return out


def _pascal_power(p: int, M: int, e: int) -> list[list[int]]:
    """P^e mod p, P_ij = binom(j, i), by repeated multiplication."""
    from math import comb
    P = [[comb(j, i) % p for j in range(M)] for i in range(M)]
    C = [[1 if i == j else 0 for j in range(M)] for i in range(M)]
    for _ in range(e):
        C = [[sum(C[i][t] * P[t][j] for t in range(M)) % p for j in range(M)] for i in range(M)]
    return C


def faure_base(r: int) -> int:
    return smallest_prime_at_least(r)


def faure_unit(n: int, r: int, first: int = 1) -> np.ndarray:
    p = faure_base(r)
    M = max_digits(p)
    out = np.empty((n, r))
    for d in range(r):
        C = _pascal_power(p, M, d)
        for i in range(n):
            kd = digits(first + i, p, M)
            y = [sum(C[a][j] * kd[j] for j in range(M)) % p for a in range(M)]
            out[i, d] = _value(y, p)
    return out


def to_box(unit: np.ndarray, half: np.ndarray) -> np.ndarray:
    """float32 box coordinates u = R_d (2 phi - 1)."""
    return (half[None, :] * (2.0 * unit - 1.0)).astype(np.float32)


def nodes(kind: str, n: int, r: int, half: np.ndarray, first: int = 1) -> np.ndarray:
    unit = halton_unit(n, r, first) if kind == "halton" else faure_unit(n, r, first)
    return to_box(unit, half)
