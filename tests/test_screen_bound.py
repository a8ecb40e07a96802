"""The error bound of the screen's Gram product, checked on the CPU.

The tensor-core screen compares |u_i|^2 + |u_s|^2 - 2 G with a threshold widened by a bound
of |G - u_i . u_s|, G computed from rounded copies of the coordinates:

* BF16 copies of u: |dG| <= 2^-6 |u_i| |u_s|;
* e4m3 copies of s u (s the largest power of two with 8 s max R <= 448):
  |dG| <= 0.14 |u_i| |u_s| + 1.07 delta sqrt(K) (|u_i| + |u_s|) + K delta^2,
  delta = 2^-10 / s, K the number of coordinates.

Here the copies are made with torch's own float conversions (round to nearest even, the
rounding of the device conversions) and the products summed exactly in float64, so the
tests bound the rounding of the operands; the bounds keep room for the accumulation inside
the tensor core (2^-9 relative per instruction for e4m3).  Cases: uniform box coordinates at
the workloads' half-width and at 8 times it (a learned box), coordinates at the rounding
midpoints of the format (the largest relative error, all of one sign), and coordinates in
the subnormal range of e4m3.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def fp8_scale(rmax: float) -> float:
    """The largest power of two s with 8 s rmax <= 448 (as the library chooses it)."""
    s = 1.0
    while s * 8.0 * rmax * 2.0 <= 448.0 and s < 1048576.0:
        s *= 2.0
    while s * 8.0 * rmax > 448.0 and s > 1.0 / 1048576.0:
        s *= 0.5
    return s


def e4m3(x: np.ndarray, s: float) -> np.ndarray:
    q = torch.from_numpy((s * x).astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.all(np.isfinite(q))
    return q / s


def bf16(x: np.ndarray) -> np.ndarray:
    return torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def fp8_bound(a: np.ndarray, b: np.ndarray, s: float) -> np.ndarray:
    K = a.shape[-1]
    delta = 2.0 ** -10 / s
    na, nb = np.linalg.norm(a, axis=-1), np.linalg.norm(b, axis=-1)
    return 0.14 * na * nb + 1.07 * delta * math.sqrt(K) * (na + nb) + K * delta * delta


def check_fp8(a: np.ndarray, b: np.ndarray, R: float) -> float:
    """Largest |dG| / bound over the rows of a and b; the accumulation allowance
    (2^-9 |a||b|) is left out of the comparison, so a ratio <= 1 keeps it in reserve."""
    s = fp8_scale(R)
    g = np.einsum("ij,ij->i", a, b)
    gq = np.einsum("ij,ij->i", e4m3(a, s), e4m3(b, s))
    bound = fp8_bound(a, b, s) - 2.0 ** -9 * np.linalg.norm(a, axis=-1) * np.linalg.norm(b, axis=-1)
    return float(np.max(np.abs(gq - g) / bound))


@pytest.mark.parametrize("R", [0.3, 2.4])
@pytest.mark.parametrize("K", [64, 128, 512, 1024])
def test_fp8_bound_uniform_box(R, K):
    rng = np.random.default_rng(K + int(10 * R))
    a = rng.uniform(-R, R, (400, K))
    b = rng.uniform(-R, R, (400, K))
    assert check_fp8(a, b, R) <= 1.0
    assert check_fp8(a, a, R) <= 1.0   # self products: every error of one sign


@pytest.mark.parametrize("K", [128, 1024])
def test_fp8_bound_at_rounding_midpoints(K):
    # s u at (1 + 2^-4) 2^e, halfway between two e4m3 codes: the largest relative rounding
    # (2^-4 / (1 + 2^-4)), of one sign for every coordinate when a = b
    R = 0.3
    s = fp8_scale(R)
    rng = np.random.default_rng(K)
    e = rng.integers(-4, 5, (50, K))
    sign = rng.choice([-1.0, 1.0], (50, K))
    a = sign * (1.0 + 2.0 ** -4) * np.exp2(e) / s
    a = np.clip(a, -R, R)
    assert check_fp8(a, a, R) <= 1.0
    b = a * (1.0 + 2.0 ** -5)   # the other operand a little off its own midpoint
    assert check_fp8(a, b, R) <= 1.0


@pytest.mark.parametrize("K", [128, 1024])
def test_fp8_bound_subnormal_range(K):
    # s u below the smallest normal e4m3 value (2^-6): absolute rounding up to 2^-10 / s
    R = 0.3
    s = fp8_scale(R)
    rng = np.random.default_rng(3 + K)
    a = rng.uniform(-(2.0 ** -6), 2.0 ** -6, (200, K)) / s
    b = rng.uniform(-(2.0 ** -6), 2.0 ** -6, (200, K)) / s
    assert check_fp8(a, b, R) <= 1.0
    assert check_fp8(a, a, R) <= 1.0
    # mixed: one operand in the box, the other tiny
    c = rng.uniform(-R, R, (200, K))
    assert check_fp8(c, a, R) <= 1.0
    # subnormal ties that round away from zero ((k + 1/2) 2^-9 with k odd goes to k + 1):
    # every self product's error 2 a delta + delta^2 of one sign, near the bound's delta terms
    k = rng.choice([1.0, 3.0, 5.0], (50, K))
    t = (k + 0.5) * 2.0 ** -9 / s * rng.choice([-1.0, 1.0], (50, K))
    assert check_fp8(t, t, R) <= 1.0


def test_fp8_scale_leaves_room_for_a_learned_box():
    for R in (0.05, 0.3, 1.0, 4.0):
        s = fp8_scale(R)
        assert 8.0 * s * R <= 448.0 < 16.0 * s * R
        x = np.array([8.0 * R, -8.0 * R])
        assert np.all(np.isfinite(e4m3(x, s)))


@pytest.mark.parametrize("K", [64, 1024])
def test_bf16_bound(K):
    rng = np.random.default_rng(11 + K)
    R = 0.3
    a = rng.uniform(-R, R, (400, K))
    b = rng.uniform(-R, R, (400, K))
    for x, y in ((a, b), (a, a)):
        g = np.einsum("ij,ij->i", x, y)
        gq = np.einsum("ij,ij->i", bf16(x), bf16(y))
        bound = 2.0 ** -6 * np.linalg.norm(x, axis=-1) * np.linalg.norm(y, axis=-1)
        assert np.max(np.abs(gq - g) / bound) <= 0.5   # half the bound left for accumulation
