"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests re-types the oracle's own formulas: they use closed forms,
invariants, special cases and an independent brute-force enumerator written
from the paper's equations with exact rational arithmetic (``fractions``), on
tiny inputs.  Each is chosen so that a plausible slip in the oracle (a dropped
line sum, a wrong sign or axis, a transposed index, an off-by-one in a
threshold) fails at least one of them; ``test_oracle_mutants.py`` checks that
claim by planting such slips in a copy of the oracle.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import phantoms

MEAN, SIGMA, ENTROPY, OKADA, OURS = 0, 1, 2, 3, 4
OURS_CROSS7, OURS_CUBE = 5, 6
SIGMA_LOCAL = 7


# --------------------------------------------------------------------------------------
# independent brute force: the equations of the paper, with exact fractions
# --------------------------------------------------------------------------------------

class Brute:
    """Direct enumeration of Eq. 2-7 on a tiny volume, in exact rationals."""

    def __init__(self, vol):
        self.vol = vol.astype(np.int64)
        self.nz, self.ny, self.nx = vol.shape
        vals = self.vol.reshape(-1)
        n = vals.size
        # population variance of the whole volume, exactly
        self.var = Fraction(int((vals * vals).sum()), n) - Fraction(int(vals.sum()), n) ** 2

    def P(self, x, y, z):
        # the volume's border value is repeated outside (clamp to edge)
        x = min(max(x, 0), self.nx - 1)
        y = min(max(y, 0), self.ny - 1)
        z = min(max(z, 0), self.nz - 1)
        return int(self.vol[z, y, x])

    def avg_cluster(self, r, cx, cy, cz):
        """Eq. 2 with Eq. 3: S = 1/(3M) (x-line + y-line + z-line of M voxels)."""
        M = 2 * r + 1
        acc = 0
        for i in range(M):
            di = i - (M - 1) // 2
            acc += self.P(cx + di, cy, cz) + self.P(cx, cy + di, cz) + self.P(cx, cy, cz + di)
        return Fraction(acc, 3 * M)

    @staticmethod
    def rnd(a):
        return math.floor(a + Fraction(1, 2))

    def ours(self, r, d, T, x, y, z):
        centres = [(x, y, z)] + [(x + sx * d, y + sy * d, z + sz * d)
                                 for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
        A = sum((self.avg_cluster(r, *c) for c in centres), Fraction(0)) / 9
        if self.P(x, y, z) >= T and A >= T:
            return self.rnd(A)
        return 0

    def ours_layout(self, layout, r, d, T, x, y, z):
        """The paper's combination (the mean of the nine cluster averages at the
        centre and the corners (+-d, +-d, +-d)) over other cluster shapes:
        'cross' = the centre and its axis cross of arm r, 'cube' = the M^3 cube."""
        centres = [(x, y, z)] + [(x + sx * d, y + sy * d, z + sz * d)
                                 for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
        avgs = []
        for cx, cy, cz in centres:
            if layout == "cross":
                vals = [self.P(cx, cy, cz)]
                for t in range(1, r + 1):
                    vals += [self.P(cx + t, cy, cz), self.P(cx - t, cy, cz), self.P(cx, cy + t, cz),
                             self.P(cx, cy - t, cz), self.P(cx, cy, cz + t), self.P(cx, cy, cz - t)]
            else:
                vals = self.cube(r, cx, cy, cz)
            avgs.append(Fraction(sum(vals), len(vals)))
        A = sum(avgs, Fraction(0)) / 9
        if self.P(x, y, z) >= T and A >= T:
            return self.rnd(A)
        return 0

    def cube(self, r, x, y, z):
        return [self.P(x + i, y + j, z + k) for k in range(-r, r + 1)
                for j in range(-r, r + 1) for i in range(-r, r + 1)]

    def mean(self, r, T, x, y, z):
        c = self.cube(r, x, y, z)
        A = Fraction(sum(c), len(c))
        return self.rnd(A) if (self.P(x, y, z) >= T and A >= T) else 0

    def sigma(self, r, k, T, x, y, z):
        # Lee's sigma filter: values within k sigma of the centre value (closed band)
        P0 = self.P(x, y, z)
        sel = [v for v in self.cube(r, x, y, z) if (v - P0) ** 2 <= k * k * self.var]
        A = Fraction(sum(sel), len(sel))
        return self.rnd(A) if (P0 >= T and A >= T) else 0

    def sigma_local(self, r, k, T, x, y, z):
        # Lee's original: the band uses the population variance of the cube itself
        P0 = self.P(x, y, z)
        c = self.cube(r, x, y, z)
        var = Fraction(sum(v * v for v in c), len(c)) - Fraction(sum(c), len(c)) ** 2
        sel = [v for v in c if (v - P0) ** 2 <= k * k * var]
        A = Fraction(sum(sel), len(sel))
        return self.rnd(A) if (P0 >= T and A >= T) else 0

    def okada(self, r, td, T, x, y, z):
        P0 = self.P(x, y, z)
        nb = [P0]
        for t in range(1, r + 1):
            for o in ((t, 0, 0), (-t, 0, 0), (0, t, 0), (0, -t, 0), (0, 0, t), (0, 0, -t)):
                nb.append(self.P(x + o[0], y + o[1], z + o[2]))
        if td is None:   # default reading: |P0 - Pi| <= sigma
            sel = [v for v in nb if (P0 - v) ** 2 <= self.var]
        else:
            sel = [v for v in nb if abs(P0 - v) < td]
        if not sel:
            return 0
        A = Fraction(sum(sel), len(sel))
        return self.rnd(A) if (P0 >= T and A >= T) else 0


@pytest.mark.parametrize("dims,dt,seed", [((4, 5, 6), "u8", 51), ((6, 4, 5), "u16", 52), ((5, 6, 4), "u16", 53)])
@pytest.mark.parametrize("mode", ["none", "otsu", "fixed"])
def test_brute_force_cluster_variants(dims, dt, seed, mode):
    vol = phantoms.random_volume(dims, seed, dt)
    T, cfg = _fixed_T(vol, mode, seed)
    b = Brute(vol)
    st = oracle.stats(vol)
    nx, ny, nz = dims
    for r in (0, 1, 2):
        prm = oracle.derive_params(st, r, cfg)
        for d in (1, 0, 2):
            for f, layout in ((OURS_CROSS7, "cross"), (OURS_CUBE, "cube")):
                got = oracle.filter_volume(vol, f, r, params=dict(prm, offset=d))
                for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
                    assert got[z, y, x] == b.ours_layout(layout, r, d, T, x, y, z), (layout, r, d, x, y, z)


@pytest.mark.parametrize("dims,dt,seed", [((4, 5, 6), "u8", 71), ((6, 4, 5), "u16", 72), ((5, 5, 5), "u8", 73)])
@pytest.mark.parametrize("mode", ["none", "otsu", "fixed"])
def test_brute_force_sigma_local(dims, dt, seed, mode):
    vol = phantoms.random_volume(dims, seed, dt)
    T, cfg = _fixed_T(vol, mode, seed)
    b = Brute(vol)
    st = oracle.stats(vol)
    nx, ny, nz = dims
    for r in (0, 1, 2):
        for k in (1, 2, 3):
            prm = dict(oracle.derive_params(st, r, cfg), k=k)
            got = oracle.filter_volume(vol, SIGMA_LOCAL, r, params=prm)
            for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
                assert got[z, y, x] == b.sigma_local(r, k, T, x, y, z), (r, k, x, y, z)


@pytest.mark.parametrize("seed", range(6))
def test_sigma_local_is_global_when_the_cube_is_the_volume(seed):
    """On a 3^3 volume the centre voxel's cube at r = 1 is the whole volume, so
    its local sigma is the global one and both filters agree there."""
    vol = phantoms.random_volume((3, 3, 3), 80 + seed, "u16" if seed % 2 else "u8")
    st = oracle.stats(vol)
    for k in (1, 2):
        prm = oracle.derive_params(st, 1, oracle.Config(sigma_k=k, threshold_mode="none"))
        pt = np.array([[1, 1, 1]])
        assert oracle.filter_points(vol, SIGMA_LOCAL, 1, pt, prm)[0] == oracle.filter_points(vol, SIGMA, 1, pt, prm)[0]


@pytest.mark.parametrize("r", [1, 2])
def test_cluster_variants_spike(r):
    """A lone spike s on a background b: only the centre cluster's axis cross
    holds it (each corner centre is off every axis through it), while every
    cube of side M >= 3 around a corner at distance 1 holds it."""
    n, c, b, s = 11, 5, 100, 4000
    vol = np.full((n, n, n), b, np.uint16)
    vol[c, c, c] = s
    prm = dict(oracle.derive_params(oracle.stats(vol), r, oracle.Config(threshold_mode="none")), offset=1)
    M = 2 * r + 1
    cross = oracle.filter_volume(vol, OURS_CROSS7, r, params=prm)
    cube = oracle.filter_volume(vol, OURS_CUBE, r, params=prm)
    assert cross[c, c, c] == math.floor(b + Fraction(s - b, 9 * (6 * r + 1)) + Fraction(1, 2))
    assert cube[c, c, c] == math.floor(b + Fraction(s - b, M ** 3) + Fraction(1, 2))
    assert (oracle.filter_volume(vol, OURS_CROSS7, r, params=prm)[0] == b).all()


def _fixed_T(vol, mode, seed):
    if mode == "none":
        return 0, oracle.Config(threshold_mode="none")
    if mode == "otsu":
        return oracle.otsu_threshold(oracle.histogram(vol)), oracle.Config()
    rng = np.random.default_rng(seed)
    t = int(rng.integers(int(vol.min()), int(vol.max()) + 1))
    return t, oracle.Config(threshold_mode="fixed", threshold_value=t)


SMALL_CASES = [
    ((4, 5, 6), "u8", 11), ((6, 4, 5), "u16", 12), ((7, 5, 4), "u8", 13),
    ((5, 6, 7), "u16", 14), ((8, 6, 5), "u8", 15),
]


@pytest.mark.parametrize("dims,dt,seed", SMALL_CASES)
@pytest.mark.parametrize("mode", ["none", "otsu", "fixed"])
def test_brute_force_mean_ours_okada(dims, dt, seed, mode):
    vol = phantoms.random_volume(dims, seed, dt)
    T, cfg = _fixed_T(vol, mode, seed)
    b = Brute(vol)
    st = oracle.stats(vol)
    nx, ny, nz = dims
    for r in (0, 1, 2, 3):
        prm = oracle.derive_params(st, r, cfg)
        assert prm["T"] == T
        for d in (1, 0, 2) if r <= 1 else (1,):
            prm_d = dict(prm, offset=d)
            got = oracle.filter_volume(vol, OURS, r, params=prm_d)
            for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
                assert got[z, y, x] == b.ours(r, d, T, x, y, z), ("ours", r, d, x, y, z)
        got = oracle.filter_volume(vol, MEAN, r, params=prm)
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            assert got[z, y, x] == b.mean(r, T, x, y, z), ("mean", r, x, y, z)
        # Okada with the default T_d (reading: |d| <= sigma) and with explicit ones
        got = oracle.filter_volume(vol, OKADA, r, params=prm)
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            assert got[z, y, x] == b.okada(r, None, T, x, y, z), ("okada", r, x, y, z)
        for td in (0, 1, 37):
            got = oracle.filter_volume(vol, OKADA, r, params=dict(prm, td=td))
            for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
                assert got[z, y, x] == b.okada(r, td, T, x, y, z), ("okada", r, td, x, y, z)


@pytest.mark.parametrize("dims,dt,seed", SMALL_CASES[:3])
@pytest.mark.parametrize("mode", ["none", "otsu"])
@pytest.mark.parametrize("k", [1, 2])
def test_brute_force_sigma(dims, dt, seed, mode, k):
    # a smoother volume so that the band actually selects
    vol = phantoms.random_volume(dims, seed, dt, p_extreme=0.3)
    T, cfg = _fixed_T(vol, mode, seed)
    cfg.sigma_k = k
    b = Brute(vol)
    st = oracle.stats(vol)
    nx, ny, nz = dims
    for r in (0, 1, 2):
        prm = oracle.derive_params(st, r, cfg)
        got = oracle.filter_volume(vol, SIGMA, r, params=prm)
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            assert got[z, y, x] == b.sigma(r, k, T, x, y, z), ("sigma", r, x, y, z)


@pytest.mark.parametrize("dims,dt,seed", [((5, 6, 7), "u16", 31), ((7, 5, 6), "u8", 32)])
@pytest.mark.parametrize("mode", ["none", "otsu"])
def test_brute_force_sigma_wide_radius(dims, dt, seed, mode):
    # r = 3 and 4: cubes of 343 and 729 taps (clamped at the faces).  Thirteen
    # neighbouring grey levels and k = 3 put most taps in the band, so band
    # counts of 256 and more occur, which the GPU tap kernel divides by
    # instead of taking a reciprocal from its table
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    base = 2000 if dt == "u16" else 120
    vol = (base + rng.integers(-6, 7, (nz, ny, nx))).astype(np.uint16 if dt == "u16" else np.uint8)
    T, cfg = _fixed_T(vol, mode, seed)
    cfg.sigma_k = 3
    b = Brute(vol)
    st = oracle.stats(vol)
    for r in (3, 4):
        prm = oracle.derive_params(st, r, cfg)
        got = oracle.filter_volume(vol, SIGMA, r, params=prm)
        most = 0
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            assert got[z, y, x] == b.sigma(r, 3, T, x, y, z), ("sigma", r, x, y, z)
            P0 = b.P(x, y, z)
            most = max(most, sum((v - P0) ** 2 <= 9 * b.var for v in b.cube(r, x, y, z)))
        assert most >= 256, (r, most)
        if mode == "otsu":
            assert 0 < np.count_nonzero(got) < got.size   # the gate splits the volume


@pytest.mark.parametrize("dims,dt,seed", SMALL_CASES)
def test_brute_force_entropy_filter(dims, dt, seed):
    """Eq. 7 in real arithmetic: the fixed-point decision must agree wherever
    the real criterion is farther from the threshold than the quantisation
    error of m rounded weights (m/2 + 1 units)."""
    vol = phantoms.random_volume(dims, seed, dt, vmax=15 if dt == "u8" else 40)
    st = oracle.stats(vol)
    N = st.N
    preal = {v: int(c) / N for v, c in enumerate(st.hist) if c > 0}
    b = Brute(vol)
    nx, ny, nz = dims
    for r in (0, 1, 2):
        m = (2 * r + 1) ** 3
        prm = oracle.derive_params(st, r, oracle.Config(threshold_mode="none"))
        te = prm["te"]
        got = oracle.filter_volume(vol, ENTROPY, r, params=prm)
        checked = 0
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            E = sum(-preal[v] * math.log2(preal[v]) for v in b.cube(r, x, y, z)) * 2 ** 22
            if abs(E - te) <= m / 2 + 1:
                continue
            want = b.P(x, y, z) if E > te else 0
            assert got[z, y, x] == want, ("entropy", r, x, y, z, E, te)
            checked += 1
        assert checked > 0.5 * nx * ny * nz


# --------------------------------------------------------------------------------------
# Eq. 1: Otsu
# --------------------------------------------------------------------------------------

def _otsu_by_definition(hist):
    """argmin over T of w0 s0^2 + w1 s1^2, class variances computed directly."""
    levels = [v for v, c in enumerate(hist) for _ in range(int(c))]
    N = len(levels)
    best = None
    for t in range(1, len(hist)):
        c0 = [v for v in levels if v < t]
        c1 = [v for v in levels if v >= t]
        if not c0 or not c1:
            continue

        def var(c):
            m = Fraction(sum(c), len(c))
            return sum((Fraction(v) - m) ** 2 for v in c) / len(c)

        sw = Fraction(len(c0), N) * var(c0) + Fraction(len(c1), N) * var(c1)
        if best is None or sw < best[0]:
            best = (sw, t)
    return best[1]


def test_otsu_two_levels():
    for a, b in ((0, 1), (20, 200), (3, 4), (100, 101), (0, 255)):
        for na, nb in ((1, 1), (5, 3), (2, 9)):
            h = np.zeros(256, np.uint64)
            h[a] = na
            h[b] = nb
            # every T in (a, b] splits the same way; ties go to the smallest
            assert oracle.otsu_threshold(h) == a + 1


def test_otsu_constant():
    for c in (0, 7, 255):
        h = np.zeros(256, np.uint64)
        h[c] = 10
        assert oracle.otsu_threshold(h) == c
    h = np.zeros(65536, np.uint64)
    h[65535] = 3
    assert oracle.otsu_threshold(h) == 65535


@pytest.mark.parametrize("seed", range(6))
def test_otsu_random_histograms_match_definition(seed):
    rng = np.random.default_rng(seed)
    h = np.zeros(256, np.uint64)
    levels = rng.choice(40, size=rng.integers(2, 8), replace=False) * 3
    for v in levels:
        h[v] = rng.integers(1, 6)
    assert oracle.otsu_threshold(h) == _otsu_by_definition(h)


def test_otsu_bimodal_between_modes():
    vol = phantoms.ellipsoid_phantom((32, 32, 32), 5, "u8", background=20, lo=180, hi=200, sigma=5)
    T = oracle.otsu_threshold(oracle.histogram(vol))
    assert 40 < T < 180


# --------------------------------------------------------------------------------------
# sigma band, Okada default, fixed-point log2 and entropy weights
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("k", [1, 2, 3])
def test_sigma_band_is_floor_of_k_sigma(seed, k):
    vol = phantoms.random_volume((9, 7, 5), seed, "u16" if seed % 2 else "u8")
    st = oracle.stats(vol)
    v = vol.astype(np.int64).reshape(-1)
    var = Fraction(int((v * v).sum()), v.size) - Fraction(int(v.sum()), v.size) ** 2
    d = oracle.sigma_band(st.N, st.S, st.Q, k)
    assert d * d <= k * k * var < (d + 1) * (d + 1)
    td = oracle.okada_td_default(st.N, st.S, st.Q)
    assert (td - 1) ** 2 <= var < td * td
    # and against numpy's population standard deviation
    assert abs(d - math.floor(k * float(np.std(v)))) <= 1


def test_log2_fixed_against_math():
    F = oracle.LOG2_FRAC_BITS
    for k in range(0, 40):
        assert oracle.log2_fixed(1 << k) == k << F
    rng = np.random.default_rng(0)
    for x in list(range(1, 300)) + [int(v) for v in rng.integers(1, 1 << 40, 300)]:
        got = oracle.log2_fixed(x) / 2 ** F
        assert abs(got - math.log2(x)) < 2.0 ** (-F + 2), x


def test_entropy_weights_against_real_terms():
    rng = np.random.default_rng(3)
    h = rng.integers(0, 5000, 256).astype(np.uint64)
    h[rng.integers(0, 256, 40)] = 0
    w = oracle.entropy_weights(h)
    N = int(h.sum())
    for v in range(256):
        if h[v] == 0:
            assert w[v] == 0
            continue
        p = int(h[v]) / N
        real = -p * math.log2(p) * 2 ** 22
        assert abs(int(w[v]) - real) <= 0.5 + 1e-6, (v, int(w[v]), real)


def test_entropy_weights_closed_forms():
    # p = 1: no information; p = 1/2 and 1/4: -p log2 p = 1/2 exactly
    h = np.zeros(256, np.uint64)
    h[9] = 17
    assert oracle.entropy_weights(h)[9] == 0
    h = np.zeros(256, np.uint64)
    h[1] = h[2] = 8
    assert list(oracle.entropy_weights(h)[[1, 2]]) == [1 << 21, 1 << 21]
    h = np.zeros(256, np.uint64)
    h[[0, 5, 6, 7]] = 4
    assert all(oracle.entropy_weights(h)[[0, 5, 6, 7]] == 1 << 21)


def test_entropy_threshold_equiprobable_levels():
    """With 2^k equally frequent levels every kernel has the same criterion,
    which equals the expectation: E > T_e never holds and the output is 0."""
    for k in (1, 2, 3):
        vals = np.arange(1 << k, dtype=np.uint8) * 7 + 3
        vol = np.resize(vals, 4 * 4 * 8).reshape(8, 4, 4)
        st = oracle.stats(vol)
        for r in (0, 1):
            prm = oracle.derive_params(st, r, oracle.Config(threshold_mode="none"))
            m = (2 * r + 1) ** 3
            assert prm["te"] == m * int(prm["w"][3])
            assert not oracle.filter_volume(vol, ENTROPY, r, params=prm).any()


# --------------------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("dt,c", [("u8", 0), ("u8", 77), ("u8", 255), ("u16", 4095), ("u16", 65535)])
def test_constant_volume(dt, c):
    vol = np.full((5, 6, 7), c, phantoms.dtype_of(dt))
    st = oracle.stats(vol)
    for r in (0, 1, 2):
        prm = oracle.derive_params(st, r)
        assert prm["T"] == c
        for f in (MEAN, SIGMA, OKADA, OURS, OURS_CROSS7, OURS_CUBE, SIGMA_LOCAL):
            assert (oracle.filter_volume(vol, f, r, params=prm) == c).all(), (f, r)
        # all weights are 0, so the criterion is 0 and 0 > T_e = 0 fails
        assert not oracle.filter_volume(vol, ENTROPY, r, params=prm).any()


@pytest.mark.parametrize("dt", ["u8", "u16"])
def test_radius_zero_identity(dt):
    vol = phantoms.random_volume((6, 5, 7), 21, dt)
    st = oracle.stats(vol)
    prm = oracle.derive_params(st, 0, oracle.Config(threshold_mode="none"))
    for f in (MEAN, SIGMA, OKADA):
        assert (oracle.filter_volume(vol, f, 0, params=prm) == vol).all(), f
    assert (oracle.filter_volume(vol, ENTROPY, 0, params=dict(prm, te=-1)) == vol).all()
    assert (oracle.filter_volume(vol, OURS, 0, params=dict(prm, offset=0)) == vol).all()


def test_radius_zero_ours_is_centre_and_corners():
    vol = phantoms.random_volume((6, 6, 6), 22, "u8")
    prm = oracle.derive_params(oracle.stats(vol), 0, oracle.Config(threshold_mode="none"))
    out = oracle.filter_volume(vol, OURS, 0, params=prm)
    v = vol.astype(np.int64)
    for z, y, x in itertools.product(range(1, 5), repeat=3):
        s = v[z, y, x] + sum(v[z + a, y + b, x + c] for a in (-1, 1) for b in (-1, 1) for c in (-1, 1))
        assert out[z, y, x] == (2 * s + 9) // 18


@pytest.mark.parametrize("r", [1, 2])
def test_linear_ramp_interior(r):
    """Symmetric windows reproduce an affine ramp exactly (mean and ours)."""
    nx, ny, nz = 14, 13, 12
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vol = (100 + 3 * x + 5 * y + 7 * z).astype(np.uint16)
    prm = oracle.derive_params(oracle.stats(vol), r, oracle.Config(threshold_mode="none"))
    h = r + 1
    for f in (MEAN, OURS):
        out = oracle.filter_volume(vol, f, r, params=prm)
        sl = (slice(h, nz - h), slice(h, ny - h), slice(h, nx - h))
        assert (out[sl] == vol[sl]).all(), f


@pytest.mark.parametrize("r", [1, 2, 3])
def test_single_spike(r):
    """A lone spike of height s on background b: only the central cluster S_0
    sees it (three times, once per line), so ours gives b + 3(s-b)/(27M); the
    mean gives b + (s-b)/M^3; sigma and Okada keep the spike untouched when it
    lies outside their bands (the spot noise the paper's Fig. 3 shows)."""
    n = 2 * (r + 2) + 3
    b, s = 20, 250
    vol = np.full((n, n, n), b, np.uint8)
    c = n // 2
    vol[c, c, c] = s
    M = 2 * r + 1
    prm = oracle.derive_params(oracle.stats(vol), r, oracle.Config(threshold_mode="none"))
    ours = oracle.filter_volume(vol, OURS, r, params=prm)
    assert ours[c, c, c] == math.floor(b + Fraction(3 * (s - b), 27 * M) + Fraction(1, 2))
    mean = oracle.filter_volume(vol, MEAN, r, params=prm)
    assert mean[c, c, c] == math.floor(b + Fraction(s - b, M ** 3) + Fraction(1, 2))
    assert prm["delta"] < s - b and prm["td"] <= s - b
    assert oracle.filter_volume(vol, SIGMA, r, params=prm)[c, c, c] == s
    assert oracle.filter_volume(vol, OKADA, r, params=prm)[c, c, c] == s


def _step_volume(a, b, k, nx=16, ny=9, nz=8, axis=0):
    g = np.where(np.arange(nx) < k, a, b)
    vol = np.broadcast_to(g[None, None, :], (nz, ny, nx)).astype(np.uint8)
    return np.ascontiguousarray(np.moveaxis(vol, 2, 2 - axis)) if axis else vol.copy()


@pytest.mark.parametrize("r", [1, 2])
def test_step_edge(r):
    """Step edge a | b along x at x = k: the output depends on x only; mean and
    ours follow the 1D tap counts; sigma and Okada keep the edge exactly when
    the step exceeds their bands."""
    # an off-centre edge, so that the population sigma (|a-b| sqrt(p(1-p)))
    # leaves the step outside both bands
    a, b, k, nx = 30, 200, 4, 16
    vol = _step_volume(a, b, k, nx=nx)
    M = 2 * r + 1
    prm = oracle.derive_params(oracle.stats(vol), r, oracle.Config(threshold_mode="none"))

    def g(x):
        x = min(max(x, 0), nx - 1)
        return a if x < k else b

    def line(cx):  # x-line of the cluster plus y- and z-lines, which are constant in x
        return sum(g(cx + i) for i in range(-r, r + 1)) + 2 * M * g(cx)

    for f in (MEAN, OURS, SIGMA, OKADA):
        out = oracle.filter_volume(vol, f, r, params=prm)
        assert (out == out[:1, :1, :]).all(), f
        assert prm["delta"] < b - a and prm["td"] <= b - a
        prof = out[0, 0, :].astype(int)
        for x in range(nx):
            if f == MEAN:
                want = math.floor(Fraction(sum(g(x + i) for i in range(-r, r + 1)), M) + Fraction(1, 2))
            elif f == OURS:
                U = line(x) + 4 * line(x - 1) + 4 * line(x + 1)
                want = math.floor(Fraction(U, 27 * M) + Fraction(1, 2))
            else:
                want = g(x)
            assert prof[x] == want, (f, x, prof[x], want)


@pytest.mark.parametrize("axis", [1, 2])
def test_step_edge_other_axes(axis):
    """The same edge turned onto the y and z axes of a non-cubic volume gives the
    same profile (catches a transposed index or a per-axis slip)."""
    r = 1
    ref = _step_volume(30, 200, 8, nx=16, ny=16, nz=16)
    vol = np.ascontiguousarray(np.swapaxes(ref, 2, 2 - axis))
    pr = oracle.derive_params(oracle.stats(ref), r, oracle.Config(threshold_mode="none"))
    for f in (MEAN, OURS, SIGMA, OKADA, ENTROPY):
        a = oracle.filter_volume(ref, f, r, params=pr)
        b = oracle.filter_volume(vol, f, r, params=pr)
        assert (np.swapaxes(a, 2, 2 - axis) == b).all(), f


def _transforms():
    for perm in itertools.permutations(range(3)):
        for flips in itertools.product((False, True), repeat=3):
            yield perm, flips


def _apply(vol, perm, flips):
    v = np.transpose(vol, perm)
    for ax, fl in enumerate(flips):
        if fl:
            v = np.flip(v, axis=ax)
    return np.ascontiguousarray(v)


@pytest.mark.parametrize("dt", ["u8", "u16"])
def test_symmetry_48(dt):
    """Every kernel and the clamp-to-edge border are symmetric under the 48
    axis permutations and flips of the cube, so the filters commute with them."""
    vol = phantoms.random_volume((6, 6, 6), 31, dt, p_extreme=0.2)
    st = oracle.stats(vol)
    outs = {}
    for f in range(10):
        # 9: the local entropy filter (id 8) on a threshold inside the cubes' range of entropies
        cfg = oracle.Config(entropy_local_te=int(4.3 * (1 << oracle.ENTROPY_W_BITS))) if f == 9 else None
        prm = oracle.derive_params(st, 1, cfg)
        outs[f] = (prm, oracle.filter_volume(vol, min(f, 8), 1, params=prm))
    assert 0 < np.count_nonzero(outs[9][1]) < np.count_nonzero(outs[8][1])
    for perm, flips in _transforms():
        tv = _apply(vol, perm, flips)
        for f in range(10):
            prm, ref = outs[f]
            got = oracle.filter_volume(tv, min(f, 8), 1, params=prm)
            assert (got == _apply(ref, perm, flips)).all(), (f, perm, flips)


def test_roi_is_crop_of_full():
    vol = phantoms.random_volume((11, 9, 10), 41, "u16")
    st = oracle.stats(vol)
    for f in range(5):
        prm = oracle.derive_params(st, 2)
        full = oracle.filter_volume(vol, f, 2, params=prm)
        roi = (2, 1, 3, 5, 6, 4)
        got = oracle.filter_volume(vol, f, 2, params=prm, roi=roi)
        x0, y0, z0, bx, by, bz = roi
        assert (got == full[z0:z0 + bz, y0:y0 + by, x0:x0 + bx]).all()
        pts = np.array([[0, 0, 0], [10, 8, 9], [5, 4, 3], [x0, y0, z0]])
        vals = oracle.filter_points(vol, f, 2, pts, prm)
        assert [int(full[z, y, x]) for x, y, z in pts] == list(vals)


# --------------------------------------------------------------------------------------
# image entropy (Fig. 4 measure)
# --------------------------------------------------------------------------------------

def test_image_entropy_closed_forms():
    h = np.zeros(256, np.uint64)
    h[5] = 100
    assert oracle.image_entropy(h) == 0.0
    for k in range(1, 9):
        h = np.zeros(256, np.uint64)
        h[: 1 << k] = 3
        assert abs(oracle.image_entropy(h) - k) < 1e-12
    for n1, n2 in ((1, 3), (7, 9), (1, 1000)):
        h = np.zeros(65536, np.uint64)
        h[0], h[65535] = n1, n2
        p = n1 / (n1 + n2)
        want = -p * math.log2(p) - (1 - p) * math.log2(1 - p)
        assert abs(oracle.image_entropy(h) - want) < 1e-12


def test_stats_moments():
    vol = phantoms.random_volume((13, 7, 5), 51, "u16")
    st = oracle.stats(vol)
    v = vol.astype(np.int64).reshape(-1)
    assert st.N == v.size and st.S == int(v.sum()) and st.Q == int((v * v).sum())
    assert st.minv == int(v.min()) and st.maxv == int(v.max())
    assert (st.hist == np.bincount(v, minlength=65536)).all()
