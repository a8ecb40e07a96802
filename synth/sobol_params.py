"""Sobol generator parameters and scramble draws (inputs, not method arithmetic).

A Sobol sequence needs, per dimension, a primitive polynomial over GF(2) and initial
direction integers m_1..m_s (odd, m_k < 2^k); the paper takes them from Joe--Kuo
tables (Appendix A, "Sobol Sequence").  No such table ships with this project, so this
module produces an equivalent table: primitive polynomials enumerated by degree (and by
their coefficient word within a degree) and initial m_k drawn from a seeded generator.
Dimension 1 is the van der Corput dimension (identity generator matrix).

Packed layout, one row of ``SOBOL_POLY_WORDS`` uint32 per dimension:
    word 0      s, the polynomial degree (0 marks the identity dimension)
    word 1      a, the inner coefficients a_1..a_{s-1} with a_1 as the most
                significant bit (the polynomial is x^s + a_1 x^{s-1} + ... + a_{s-1} x + 1)
    words 2..   m_1..m_s

Affine (Matousek) scramble draws, one row of ``SOBOL_SCRAMBLE_WORDS`` uint32 per
dimension:
    words 0..31 rows k = 1..32 of a lower-triangular, unit-diagonal 32x32 GF(2) matrix.
                Row k acts on output digit k (weight 2^-k, stored at bit 32-k) and has
                bits only for input digits j <= k, i.e. bits >= 32-k; bit 32-k is set.
    word 32     the digital shift e (one uint32, digit k at bit 32-k).
"""
from __future__ import annotations

import numpy as np

SOBOL_POLY_WORDS = 16
SOBOL_SCRAMBLE_WORDS = 33
SOBOL_MAX_DIM = 1 + 1 + 2 + 2 + 6 + 6 + 18 + 16 + 48 + 60 + 176 + 144 + 630 + 756  # degrees 1..14


def _prime_factors(v: int) -> list[int]:
    out, p = [], 2
    while p * p <= v:
        if v % p == 0:
            out.append(p)
            while v % p == 0:
                v //= p
        p += 1
    if v > 1:
        out.append(v)
    return out


def _polymulmod(a: int, b: int, p: int, deg: int) -> int:
    """Product of two GF(2) polynomials (bit k = coefficient of x^k) modulo p."""
    res = 0
    while b:
        if b & 1:
            res ^= a
        b >>= 1
        a <<= 1
        if (a >> deg) & 1:
            a ^= p
    return res


def _polypowmod(base: int, e: int, p: int, deg: int) -> int:
    res = 1
    while e:
        if e & 1:
            res = _polymulmod(res, base, p, deg)
        base = _polymulmod(base, base, p, deg)
        e >>= 1
    return res


def _is_primitive(p: int, deg: int) -> bool:
    """x has multiplicative order exactly 2^deg - 1 modulo p."""
    if not (p & 1):
        return False
    if deg == 1:
        return p == 0b11
    order = (1 << deg) - 1
    if _polypowmod(0b10, order, p, deg) != 1:
        return False
    return all(_polypowmod(0b10, order // q, p, deg) != 1 for q in _prime_factors(order))


def primitive_polynomials(count: int) -> list[tuple[int, int]]:
    """First ``count`` primitive polynomials as (degree s, inner coefficient word a)."""
    out: list[tuple[int, int]] = []
    deg = 1
    while len(out) < count:
        if deg > 14:
            raise ValueError("more dimensions requested than degree-14 polynomials cover")
        for a in range(1 << max(deg - 1, 0)):
            p = (1 << deg) | (a << 1) | 1
            if _is_primitive(p, deg):
                out.append((deg, a))
                if len(out) == count:
                    break
        deg += 1
    return out


def sobol_poly_params(r: int, seed: int) -> np.ndarray:
    """Packed generator parameters for dimensions 1..r (uint32 [r][SOBOL_POLY_WORDS])."""
    if not 1 <= r <= SOBOL_MAX_DIM:
        raise ValueError(f"r must be in [1, {SOBOL_MAX_DIM}]")
    rng = np.random.Generator(np.random.Philox(key=np.uint64(seed) ^ np.uint64(0x5B0B01)))
    out = np.zeros((r, SOBOL_POLY_WORDS), dtype=np.uint32)
    polys = primitive_polynomials(r - 1)
    for d in range(1, r):
        s, a = polys[d - 1]
        out[d, 0] = s
        out[d, 1] = a
        for k in range(1, s + 1):
            # odd and below 2^k
            out[d, 1 + k] = 2 * int(rng.integers(0, 1 << (k - 1))) + 1
    return out


def sobol_scramble_params(r: int, seed: int) -> np.ndarray:
    """Random affine scramble (uint32 [r][SOBOL_SCRAMBLE_WORDS]); see module docstring."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(seed) ^ np.uint64(0x5C4A3B1E)))
    out = np.zeros((r, SOBOL_SCRAMBLE_WORDS), dtype=np.uint32)
    raw = rng.integers(0, 1 << 32, size=(r, 33), dtype=np.uint64)
    for k in range(1, 33):
        diag = np.uint64(1) << np.uint64(32 - k)
        above = np.uint64(((1 << 32) - 1) ^ ((1 << (33 - k)) - 1))  # bits > 32-k
        out[:, k - 1] = ((raw[:, k - 1] & above) | diag).astype(np.uint32)
    out[:, 32] = raw[:, 32].astype(np.uint32)
    return out


def identity_scramble(r: int) -> np.ndarray:
    """Scramble words that leave the sequence unchanged (identity matrix, zero shift)."""
    out = np.zeros((r, SOBOL_SCRAMBLE_WORDS), dtype=np.uint32)
    for k in range(1, 33):
        out[:, k - 1] = np.uint32(1 << (32 - k))
    return out
