"""Pins of the oracle's entropy filter with local probabilities (filter id 8;
the information entropy of the kernel, paper section "Related Work"): the
fixed-point table against libm, the keep / zero decision against the entropy
of the cube computed in real numbers (libm) wherever the two are not within
the table's rounding of the threshold, a two-level cube against the binary
entropy in closed form, constant and all-distinct cubes, the noise gate and
the pass-all threshold.  The 48 symmetries are in test_oracle_pins.py."""
import math
from collections import Counter

import numpy as np
import pytest

import oracle

EL = oracle.ENTROPY_LOCAL
W = oracle.ENTROPY_W_BITS


def test_table_against_libm():
    m = 17 ** 3
    t = oracle.local_entropy_table(m)
    assert t[0] == 0 and t[1] == 0
    for c in range(2, m + 1):
        exact = (1 << W) * c * math.log2(c)
        # round to nearest, after the 40-bit logarithm's truncation (below 2^-40 on
        # log2 c, so below c 2^(22-40) on the entry); libm's error is far smaller
        assert abs(int(t[c]) - exact) <= 0.5 + c * 2.0 ** (W - 40) + 1e-6, c


def _sample(vol, x, y, z):
    nz, ny, nx = vol.shape
    return int(vol[min(max(z, 0), nz - 1), min(max(y, 0), ny - 1), min(max(x, 0), nx - 1)])


def _real_criterion(vol, r, x, y, z):
    """m 2^22 H of the clamped cube, H from libm: (m, value)."""
    vals = [_sample(vol, x + i, y + j, z + k) for k in range(-r, r + 1) for j in range(-r, r + 1)
            for i in range(-r, r + 1)]
    m = len(vals)
    H = -sum(c / m * math.log2(c / m) for c in Counter(vals).values())
    return m, m * (1 << W) * H


def _volume(dims, dt, levels, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    v = rng.integers(0, levels, (nz, ny, nx))
    if dt == "u16":
        v = v * 97 + 300          # spread the few levels over 16 bits
    return v.astype(np.uint8 if dt == "u8" else np.uint16)


@pytest.mark.parametrize("dims,dt,levels,seed", [
    ((4, 4, 4), "u8", 3, 1), ((5, 6, 7), "u8", 6, 2), ((8, 5, 4), "u16", 12, 3), ((6, 6, 6), "u8", 40, 4),
    ((7, 4, 5), "u16", 200, 5)])
@pytest.mark.parametrize("r", [0, 1, 2])
def test_decision_against_real_entropy(dims, dt, levels, seed, r):
    vol = _volume(dims, dt, levels, seed)
    st = oracle.stats(vol)
    nx, ny, nz = dims
    m = (2 * r + 1) ** 3
    for theta in (None, 0, (1 << W) // 2, (1 << W) * 2):
        prm = oracle.derive_params(st, r, oracle.Config(threshold_mode="none", entropy_local_te=theta))
        th = oracle.local_entropy_te_default(oracle.local_entropy_table(m), m) if theta is None else theta
        got = oracle.filter_volume(vol, EL, r, params=prm)
        decided = 0
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    mm, crit = _real_criterion(vol, r, x, y, z)
                    # the fixed-point criterion sums at most m + 1 table entries,
                    # each within 1/2 of its real value
                    if abs(crit - mm * th) <= mm + 2:
                        continue
                    decided += 1
                    want = int(vol[z, y, x]) if crit > mm * th else 0
                    assert int(got[z, y, x]) == want, (r, theta, x, y, z, crit, mm * th)
        if r > 0 or th != 0:        # (r = 0: every cube has H = 0, on a zero threshold)
            assert decided >= 0.8 * vol.size


@pytest.mark.parametrize("k", range(1, 28))
def test_two_level_cube_is_the_binary_entropy(k):
    """The 3^3 volume at r = 1 seen from its centre: the cube is the volume, k
    voxels at level a (the centre among them) and 27 - k at level b."""
    a, b = 200, 60
    flat = np.full(27, b, np.uint8)
    flat[13] = a
    others = [i for i in range(27) if i != 13]
    flat[others[:k - 1]] = a
    vol = flat.reshape(3, 3, 3)
    p = k / 27
    H = 0.0 if k == 27 else -(p * math.log2(p) + (1 - p) * math.log2(1 - p))
    st = oracle.stats(vol)
    for theta_bits in (0.0, 0.3, 0.5, 0.9, 0.99):
        th = int(theta_bits * (1 << W))
        prm = oracle.derive_params(st, 1, oracle.Config(threshold_mode="fixed", threshold_value=a,
                                                         entropy_local_te=th))
        got = int(oracle.filter_points(vol, EL, 1, [(1, 1, 1)], prm)[0])
        if abs(H * (1 << W) - th) <= 28:
            continue
        assert got == (a if H * (1 << W) > th else 0), (k, theta_bits, H)


def test_constant_and_distinct_cubes_and_the_gate():
    # constant: H = 0, never above a threshold >= 0; the pass-all threshold keeps P0
    vol = np.full((5, 5, 5), 77, np.uint8)
    st = oracle.stats(vol)
    prm = oracle.derive_params(st, 1, oracle.Config(threshold_mode="none"))
    assert not oracle.filter_volume(vol, EL, 1, params=prm).any()
    prm = oracle.derive_params(st, 1, oracle.Config(threshold_mode="none", entropy_local_te=-1))
    assert (oracle.filter_volume(vol, EL, 1, params=prm) == 77).all()
    # H = 0 exactly (the criterion is t[m] - t[m]): not above a zero threshold
    prm = oracle.derive_params(st, 1, oracle.Config(threshold_mode="none", entropy_local_te=0))
    assert not oracle.filter_volume(vol, EL, 1, params=prm).any()
    # all 27 values distinct: H = log2 27, above the default log2(27) / 2
    vol = (np.arange(27, dtype=np.uint16) * 11 + 5).reshape(3, 3, 3)
    st = oracle.stats(vol)
    prm = oracle.derive_params(st, 1, oracle.Config(threshold_mode="none"))
    assert int(oracle.filter_points(vol, EL, 1, [(1, 1, 1)], prm)[0]) == int(vol[1, 1, 1])
    # the gate: P0 < T gives 0 whatever the entropy
    prm = oracle.derive_params(st, 1, oracle.Config(threshold_mode="fixed", threshold_value=int(vol[1, 1, 1]) + 1))
    assert int(oracle.filter_points(vol, EL, 1, [(1, 1, 1)], prm)[0]) == 0
    # radius 0: a cube of one voxel has H = 0
    prm = oracle.derive_params(st, 0, oracle.Config(threshold_mode="none"))
    assert not oracle.filter_volume(vol, EL, 0, params=prm).any()
