"""Scrambled Sobol nodes (Appendix A, "Sobol Sequence"; scrambling per "Practical
considerations" and the MatousekAffineOwen choice named there).

Direction numbers: for a dimension with primitive polynomial
x^s + a_1 x^{s-1} + ... + a_{s-1} x + 1 and initial m_1..m_s, V_k = m_k 2^(32-k) for
k <= s and, for k > s, the Bratley--Fox recurrence
    V_k = a_1 V_{k-1} xor ... xor a_{s-1} V_{k-s+1} xor V_{k-s} xor (V_{k-s} >> s).
The identity dimension (s = 0) has V_k = 2^(32-k) (van der Corput).

Point n, dimension d: XOR of V_k over the set bits b_k of the Gray code
g(n) = n xor (n >> 1) (the appendix's x_n = b_1 (x) v_1 xor b_2 (x) v_2 xor ...).

Affine scramble: digit k of the scrambled integer is the parity of (row_k AND y) xor
digit k of the shift (a lower-triangular, unit-diagonal GF(2) matrix plus a digital
shift).  Coordinate in the box: u = R * (2 (y + 1/2) 2^-32 - 1), evaluated in float64
(the only rounding is the product with R) and then rounded to float32.
"""
from __future__ import annotations

import numpy as np


def direction_numbers(poly_row: np.ndarray) -> np.ndarray:
    """uint32 V_1..V_32 for one packed parameter row (see synth.sobol_params)."""
    s = int(poly_row[0])
    a = int(poly_row[1])
    V = [0] * 33  # 1-based
    if s == 0:
        for k in range(1, 33):
            V[k] = 1 << (32 - k)
    else:
        for k in range(1, min(s, 32) + 1):
            V[k] = int(poly_row[1 + k]) << (32 - k)
        for k in range(s + 1, 33):
            v = V[k - s] ^ (V[k - s] >> s)
            for i in range(1, s):
                if (a >> (s - 1 - i)) & 1:
                    v ^= V[k - i]
            V[k] = v & 0xFFFFFFFF
    return np.array(V[1:], dtype=np.uint64)


def sobol_integers(poly: np.ndarray, n: int, first_index: int = 0) -> np.ndarray:
    """Unscrambled Sobol integers y[i][d] (uint32) for indices first_index..+n-1."""
    r = poly.shape[0]
    idx = np.arange(first_index, first_index + n, dtype=np.uint64)
    gray = idx ^ (idx >> np.uint64(1))
    out = np.zeros((n, r), dtype=np.uint64)
    for d in range(r):
        V = direction_numbers(poly[d])
        acc = np.zeros(n, dtype=np.uint64)
        for b in range(32):
            bit = (gray >> np.uint64(b)) & np.uint64(1)
            acc ^= bit * V[b]
        out[:, d] = acc
    return out.astype(np.uint32)


def scramble(y: np.ndarray, scr: np.ndarray) -> np.ndarray:
    """Apply the affine scramble of each dimension to integers y[i][d]."""
    n, r = y.shape
    out = np.zeros((n, r), dtype=np.uint64)
    yy = y.astype(np.uint64)
    for d in range(r):
        col = yy[:, d]
        res = np.zeros(n, dtype=np.uint64)
        for k in range(1, 33):
            row = np.uint64(int(scr[d, k - 1]))
            x = col & row
            # parity of x by folding halves (x < 2^32)
            for sh in (16, 8, 4, 2, 1):
                x = x ^ (x >> np.uint64(sh))
            p = x & np.uint64(1)
            ek = (np.uint64(int(scr[d, 32])) >> np.uint64(32 - k)) & np.uint64(1)
            res |= (p ^ ek) << np.uint64(32 - k)
        out[:, d] = res
    return out.astype(np.uint32)


def to_box(y: np.ndarray, R: float) -> np.ndarray:
    """float32 box coordinates u = R (2 (y + 1/2) 2^-32 - 1)."""
    t = (y.astype(np.float64) + 0.5) * (2.0 ** -32)
    return (R * (2.0 * t - 1.0)).astype(np.float32)


def nodes(poly: np.ndarray, scr: np.ndarray | None, n: int, R: float,
          first_index: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(scrambled integers uint32 [n][r], float32 box coordinates [n][r])."""
    y = sobol_integers(poly, n, first_index)
    if scr is not None:
        y = scramble(y, scr)
    return y, to_box(y, R)
