"""Pins for the multi-scale kernel coefficients ("Second-Order Kernel Construction" and
"High-Order Kernel Construction")."""
import math
import os

import numpy as np
import pytest

from oracle import coeffs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "second_order_coefficients.txt")


def _golden():
    vals = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        name, a, b = line.split()
        vals[name] = float(b) + float(a) * math.sqrt(2.0)
    return vals


def test_second_order_matches_printed_closed_form():
    g = _golden()
    c = coeffs.kernel_coefficients(2)
    assert c[0] == pytest.approx(g["alpha"], abs=1e-13)
    assert c[1] == pytest.approx(g["beta"], abs=1e-13)
    assert c[2] == pytest.approx(g["gamma"], abs=1e-13)


def test_first_order_is_plain_kernel():
    c = coeffs.kernel_coefficients(1)
    assert c[0] == pytest.approx(1.0, abs=1e-15)
    assert abs(c[1]) < 1e-15


@pytest.mark.parametrize("N", [3, 4, 5])
def test_higher_order_conditions(N):
    """Constant matching, dt matching and elimination of (dt)^mu, mu = 3/2, 2, ...,
    checked term by term on a synthetic expansion: for any smooth u with
    L_{dt/s} u = u + (dt/s) A + sum_k C_k (dt/s)^{mu_k}, the combination must
    reproduce u + dt A exactly."""
    c = coeffs.kernel_coefficients(N)
    s = [2.0 ** j for j in range(N)]
    mus = [1.5 + 0.5 * k for k in range(N - 1)]
    rng = np.random.default_rng(N)
    u, A = rng.normal(size=2)
    Ck = rng.normal(size=N - 1)
    for dt in (0.1, 0.01, 0.37):
        comb = c[N] * u
        for j in range(N):
            tau = dt / s[j]
            comb += c[j] * (u + tau * A + sum(Ck[k] * tau ** mus[k] for k in range(N - 1)))
        assert comb == pytest.approx(u + dt * A, abs=1e-10)


def test_third_order_values():
    """N = 3 with s = (1, 2, 4), mu = (3/2, 2).  Eliminating c_3 and c_2 by hand gives
    c_2 = -2 - 6 c_1 and c_1 = -2k / (1 + 6k) with k = (1 - sqrt2) / (2 sqrt2), i.e.
    c_1 = 1 + sqrt2.  Cramer's rule is also checked against an LU solve."""
    c = coeffs.kernel_coefficients(3)
    V, d = coeffs.vandermonde(3)
    assert np.allclose(np.linalg.solve(V, d), c, rtol=0, atol=1e-12)
    assert np.linalg.norm(V @ c - d) < 1e-12
    # c_1 = 1 + sqrt(2) (from eliminating c_2, c_3 by hand)
    assert c[0] == pytest.approx(1.0 + math.sqrt(2.0), abs=1e-12)
