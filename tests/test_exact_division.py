"""The kernels round averages with multiply-high arithmetic instead of
division (Granlund and Montgomery's method).  Check, exhaustively over each
proven input range, that the method gives round-half-up exactly:
  * division by the constants 27M (the paper's filter) and M^3 (mean),
    floor((x + (D-1)/2) / D) with q = (x m) >> (32 + s), m = ceil(2^(32+s)/D),
    s the smallest shift with x_max e < 2^(32+s);
  * division by a voxel count n < 256 (sigma, Okada) with the reciprocal
    ceil(2^32 / n), for sums up to n * 65535."""
import numpy as np
import pytest


def params(D, xmax):
    for s in range(21):
        m = ((1 << (32 + s)) + D - 1) // D
        if m < (1 << 32) and (m * D - (1 << (32 + s))) * xmax < (1 << (32 + s)):
            return s, m
    raise AssertionError("no multiplier")


def check_range(D, n_max, q_of):
    step = 1 << 22
    for lo in range(0, n_max + 1, step):
        x = np.arange(lo, min(n_max, lo + step - 1) + 1, dtype=np.uint64)
        want = (2 * x + D) // (2 * D)
        assert np.array_equal(q_of(x), want), (D, lo)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["ours", "mean"])
def test_constant_divisors(r, kind):
    M = 2 * r + 1
    D = 27 * M if kind == "ours" else M ** 3
    s, m = params(D, D * 65536)
    half = (D - 1) // 2
    check_range(D, D * 65535, lambda x: (x * np.uint64(m) + np.uint64(half * m)) >> np.uint64(32 + s))


def test_reciprocal_table():
    for n in range(2, 256):
        r = ((1 << 32) + n - 1) // n
        sm = np.arange(0, n * 65535 + 1, dtype=np.uint64)
        q = ((sm + np.uint64(n >> 1)) * np.uint64(r)) >> np.uint64(32)
        assert np.array_equal(q, (2 * sm + n) // (2 * n)), n
