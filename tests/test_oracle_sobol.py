"""Pins for the oracle's Sobol nodes (Appendix A, "Sobol Sequence")."""
import numpy as np
import pytest

from oracle import sobol
from synth import sobol_poly_params, sobol_scramble_params, primitive_polynomials
from synth.sobol_params import identity_scramble, SOBOL_POLY_WORDS

NBITS = 15   # direction numbers recovered from scipy: V_1..V_15


def _scipy_direction_numbers(dim):
    qmc = pytest.importorskip("scipy.stats.qmc")
    eng = qmc.Sobol(d=dim, scramble=False, bits=32)
    pts = eng.random(2 ** NBITS)
    ints = np.round(pts * 2.0 ** 32).astype(np.uint64)
    # gray(2^(b+1) - 1) = 2^b, so that point is V_{b+1} itself
    idx = [(1 << (b + 1)) - 1 for b in range(NBITS)]
    return ints[idx, :].T, ints   # [dim][NBITS], all points


def test_engine_and_recurrence_against_scipy():
    """scipy's unscrambled Sobol (Joe--Kuo numbers) through its public API: for every
    dimension some primitive polynomial of degree <= 7 with the recovered m_1..m_s must
    reproduce V_1..V_15 through the oracle's recurrence, and the oracle's Gray-code
    engine fed those parameters must reproduce scipy's first 4096 points bit for bit."""
    dim = 24
    V, ints = _scipy_direction_numbers(dim)
    polys = primitive_polynomials(60)
    params = np.zeros((dim, SOBOL_POLY_WORDS), dtype=np.uint32)
    for d in range(1, dim):
        found = False
        for (s, a) in polys:
            row = np.zeros(SOBOL_POLY_WORDS, dtype=np.uint32)
            row[0], row[1] = s, a
            for k in range(1, s + 1):
                row[1 + k] = int(V[d, k - 1]) >> (32 - k)
            if np.array_equal(sobol.direction_numbers(row)[:NBITS], V[d]):
                params[d] = row
                found = True
                break
        assert found, f"no primitive polynomial reproduces scipy dimension {d + 1}"
    assert np.array_equal(sobol.direction_numbers(params[0])[:NBITS], V[0])
    y = sobol.sobol_integers(params, 4096)
    assert np.array_equal(y.astype(np.uint64), ints[:4096])


def test_van_der_corput_first_dimension():
    y = sobol.sobol_integers(sobol_poly_params(1, 0), 8)[:, 0]
    expect = np.array([0, 4, 6, 2, 3, 7, 5, 1], dtype=np.uint64) << np.uint64(29)
    assert np.array_equal(y.astype(np.uint64), expect)


@pytest.mark.parametrize("scrambled", [False, True])
def test_one_point_per_elementary_interval(scrambled):
    """(0, m, 1)-net property of every 1-D projection of the first 2^m points; the
    affine scramble (unit-diagonal lower-triangular matrix + shift) preserves it."""
    r, m = 40, 10
    poly = sobol_poly_params(r, 7)
    scr = sobol_scramble_params(r, 7) if scrambled else None
    y, _ = sobol.nodes(poly, scr, 1 << m, 1.0)
    cells = (y >> np.uint32(32 - m)).astype(np.int64)
    for d in range(r):
        assert np.array_equal(np.sort(cells[:, d]), np.arange(1 << m))


def test_identity_scramble_is_noop_and_scramble_changes_points():
    r = 5
    poly = sobol_poly_params(r, 3)
    y0 = sobol.sobol_integers(poly, 64)
    assert np.array_equal(sobol.scramble(y0, identity_scramble(r)), y0)
    y1 = sobol.scramble(y0, sobol_scramble_params(r, 3))
    assert not np.array_equal(y1, y0)


def test_scramble_is_affine_bijection_on_digit_prefixes():
    """Brute force on 8-bit prefixes: with a unit-diagonal lower-triangular matrix the
    top k digits of the output depend only on the top k input digits, bijectively."""
    scr = sobol_scramble_params(1, 11)
    top = np.arange(256, dtype=np.uint64) << np.uint64(24)
    out = sobol.scramble(top.astype(np.uint32)[:, None], scr)[:, 0]
    assert len(set((out >> np.uint32(24)).tolist())) == 256


def test_box_mapping_values():
    R = 0.75
    y = np.array([[0], [1 << 31], [0xFFFFFFFF]], dtype=np.uint32)
    u = sobol.to_box(y, R)[:, 0]
    assert u[0] == np.float32(R * (2.0 ** -31 * 0.5 * 2 - 1.0))
    assert u[1] == np.float32(R * 2.0 ** -32)
    assert u[2] == np.float32(R * (1.0 - 2.0 ** -32))
    assert u.dtype == np.float32


def test_polynomials_are_primitive_by_period():
    """Brute force: an LFSR with a primitive polynomial of degree s has period 2^s - 1."""
    for (s, a) in primitive_polynomials(30):
        if s > 10:
            break
        taps = (1 << s) | (a << 1) | 1
        state, period = 1, 0
        while True:
            state <<= 1
            if state >> s & 1:
                state ^= taps
            period += 1
            if state == 1:
                break
        assert period == (1 << s) - 1
