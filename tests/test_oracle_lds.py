"""Pins for the oracle's Halton and Faure node sets (oracle/lds.py): scipy's Halton through
its public API, hand-worked radical inverses, the net property of the Faure sequence, and
the coincidence of the two-dimensional base-2 Faure point set with the first two Sobol
dimensions."""
import itertools

import numpy as np
import pytest

from oracle import lds


def test_halton_matches_scipy():
    qmc = pytest.importorskip("scipy.stats.qmc")
    ref = qmc.Halton(d=7, scramble=False).random(300)
    ours = lds.halton_unit(300, 7, first=0)
    assert np.max(np.abs(ours - ref)) <= 1e-15


def test_halton_hand_values():
    h = lds.halton_unit(5, 2, first=1)
    assert h[:3, 0].tolist() == [0.5, 0.25, 0.75]          # base 2: 1, 10, 11 reversed
    assert h[0, 1] == 1 / 3 and h[1, 1] == 2 / 3
    assert h[4, 1] == pytest.approx(7 / 9, abs=1e-16)       # 5 = 12 in base 3 -> 0.21 = 2/3 + 1/9
    assert lds.first_primes(8) == [2, 3, 5, 7, 11, 13, 17, 19]
    assert lds.smallest_prime_at_least(1024) == 1031 and lds.faure_base(7) == 7 and lds.faure_base(1) == 2


@pytest.mark.parametrize("r,m", [(2, 4), (3, 3), (5, 2), (4, 2)])
def test_faure_is_a_net(r, m):
    """(0, m, r)-net in base p: among points 0 .. p^m - 1, every elementary interval
    prod_d [a_d p^-m_d, (a_d + 1) p^-m_d) with sum m_d = m holds exactly one point."""
    p = lds.faure_base(r)
    x = lds.faure_unit(p ** m, r, first=0)
    for ms in itertools.product(range(m + 1), repeat=r):
        if sum(ms) != m:
            continue
        cells = np.stack([np.floor(x[:, d] * p ** ms[d]).astype(np.int64) for d in range(r)], axis=1)
        _, counts = np.unique(cells, axis=0, return_counts=True)
        assert counts.size == p ** m and np.all(counts == 1), ms


def test_faure_first_dimension_is_van_der_corput_in_its_base():
    p = lds.faure_base(5)
    x = lds.faure_unit(30, 5, first=1)
    for k in range(1, 31):
        dig, v, s = [], 0.0, k
        while s:
            dig.append(s % p)
            s //= p
        v = sum(dd * p ** -(i + 1) for i, dd in enumerate(dig))
        assert x[k - 1, 0] == pytest.approx(v, abs=1e-15)


def test_base2_faure_equals_sobol_point_set():
    qmc = pytest.importorskip("scipy.stats.qmc")
    m = 6
    fa = lds.faure_unit(2 ** m, 2, first=0)
    so = qmc.Sobol(d=2, scramble=False).random(2 ** m)
    key = lambda a: np.round(a * 2 ** m).astype(np.int64)
    assert sorted(map(tuple, key(fa))) == sorted(map(tuple, key(so)))


def test_box_map():
    u = lds.to_box(np.array([[0.5, 0.0, 0.75]]), np.array([0.3, 2.0, 4.0]))
    assert u.dtype == np.float32 and u.tolist() == [[0.0, -2.0, 2.0]]
