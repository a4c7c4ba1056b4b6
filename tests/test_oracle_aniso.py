"""Pins of the oracle's anisotropic form (voxel spacing that differs per axis):
every filter takes a radius and a cluster offset per axis (x, y, z).  The paper's
volumes are isotropic; the reading generalises each definition axis by axis:

  * the cube of M^3 voxels (mean Eq. 4, sigma Eq. 5, entropy Eq. 7, the local
    sigma) becomes the box of Mx * My * Mz voxels, M_a = 2 r_a + 1;
  * the Okada cross (Eq. 6) has arm r_a along axis a;
  * a cluster of the paper's filter (Eq. 2-3) averages its x-, y- and z-lines of
    Mx, My and Mz voxels (the centre three times, Mx + My + Mz samples), and the
    eight diagonal clusters sit at (+-dx, +-dy, +-dz);
  * radii come from a physical extent and the spacing by rounding half up.

With equal radii and offsets every form is the isotropic one.  The pins are an
exact-rational enumerator written from these definitions, closed forms, the
axis-permutation symmetry, and the spacing rounding."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import phantoms

MEAN, SIGMA, ENTROPY, OKADA, OURS = 0, 1, 2, 3, 4
OURS_CROSS7, OURS_CUBE, SIGMA_LOCAL = 5, 6, 7


class AnisoBrute:
    """Direct enumeration of the per-axis definitions in exact rationals."""

    def __init__(self, vol, w=None):
        self.vol = vol.astype(np.int64)
        self.nz, self.ny, self.nx = vol.shape
        vals = self.vol.reshape(-1)
        n = vals.size
        self.var = Fraction(int((vals * vals).sum()), n) - Fraction(int(vals.sum()), n) ** 2
        self.w = w

    def P(self, x, y, z):
        return int(self.vol[min(max(z, 0), self.nz - 1), min(max(y, 0), self.ny - 1), min(max(x, 0), self.nx - 1)])

    @staticmethod
    def rnd(a):
        return math.floor(a + Fraction(1, 2))

    def box(self, r, x, y, z):
        rx, ry, rz = r
        return [self.P(x + i, y + j, z + k) for k in range(-rz, rz + 1)
                for j in range(-ry, ry + 1) for i in range(-rx, rx + 1)]

    def gate(self, x, y, z, A, T):
        return self.rnd(A) if (self.P(x, y, z) >= T and A >= T) else 0

    def centres(self, d, x, y, z):
        dx, dy, dz = d
        return [(x, y, z)] + [(x + sx * dx, y + sy * dy, z + sz * dz)
                              for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]

    def ours(self, r, d, T, x, y, z):
        rx, ry, rz = r
        avgs = []
        for cx, cy, cz in self.centres(d, x, y, z):
            lines = ([self.P(cx + t, cy, cz) for t in range(-rx, rx + 1)]
                     + [self.P(cx, cy + t, cz) for t in range(-ry, ry + 1)]
                     + [self.P(cx, cy, cz + t) for t in range(-rz, rz + 1)])
            avgs.append(Fraction(sum(lines), len(lines)))
        return self.gate(x, y, z, sum(avgs, Fraction(0)) / 9, T)

    def ours_layout(self, layout, r, d, T, x, y, z):
        avgs = []
        for cx, cy, cz in self.centres(d, x, y, z):
            if layout == "cross":
                vals = [self.P(cx, cy, cz)]
                for t in range(1, r[0] + 1):
                    vals += [self.P(cx + t, cy, cz), self.P(cx - t, cy, cz)]
                for t in range(1, r[1] + 1):
                    vals += [self.P(cx, cy + t, cz), self.P(cx, cy - t, cz)]
                for t in range(1, r[2] + 1):
                    vals += [self.P(cx, cy, cz + t), self.P(cx, cy, cz - t)]
            else:
                vals = self.box(r, cx, cy, cz)
            avgs.append(Fraction(sum(vals), len(vals)))
        return self.gate(x, y, z, sum(avgs, Fraction(0)) / 9, T)

    def mean(self, r, T, x, y, z):
        b = self.box(r, x, y, z)
        return self.gate(x, y, z, Fraction(sum(b), len(b)), T)

    def sigma(self, r, k, T, x, y, z):
        P0 = self.P(x, y, z)
        sel = [v for v in self.box(r, x, y, z) if (v - P0) ** 2 <= k * k * self.var]
        return self.gate(x, y, z, Fraction(sum(sel), len(sel)), T)

    def sigma_local(self, r, k, T, x, y, z):
        P0 = self.P(x, y, z)
        b = self.box(r, x, y, z)
        var = Fraction(sum(v * v for v in b), len(b)) - Fraction(sum(b), len(b)) ** 2
        sel = [v for v in b if (v - P0) ** 2 <= k * k * var]
        return self.gate(x, y, z, Fraction(sum(sel), len(sel)), T)

    def okada(self, r, td, T, x, y, z):
        P0 = self.P(x, y, z)
        nb = [P0]
        for a in range(3):
            for t in range(1, r[a] + 1):
                for s in (t, -t):
                    o = [0, 0, 0]
                    o[a] = s
                    nb.append(self.P(x + o[0], y + o[1], z + o[2]))
        sel = [v for v in nb if abs(P0 - v) < td]
        if not sel:
            return 0
        return self.gate(x, y, z, Fraction(sum(sel), len(sel)), T)

    def entropy(self, r, te, T, x, y, z):
        E = sum(int(self.w[v]) for v in self.box(r, x, y, z))
        P0 = self.P(x, y, z)
        return P0 if (P0 >= T and E > te) else 0


RADII = [(0, 1, 2), (2, 0, 1), (1, 2, 0), (1, 1, 0), (2, 1, 1)]
OFFSETS = [(1, 1, 1), (1, 0, 2), (2, 1, 0)]


def _T(vol, mode):
    if mode == "none":
        return 0, oracle.Config(threshold_mode="none")
    T = oracle.otsu_threshold(oracle.stats(vol).hist)
    return T, oracle.Config()


@pytest.mark.parametrize("dims,dt,seed", [((5, 4, 6), "u8", 301), ((4, 6, 5), "u16", 302)])
@pytest.mark.parametrize("mode", ["none", "otsu"])
def test_brute_force_anisotropic(dims, dt, seed, mode):
    vol = phantoms.random_volume(dims, seed, dt)
    T, cfg = _T(vol, mode)
    st = oracle.stats(vol)
    nx, ny, nz = dims
    for ri, r in enumerate(RADII):
        prm = oracle.derive_params(st, r, cfg)
        b = AnisoBrute(vol, prm["w"])
        m = (2 * r[0] + 1) * (2 * r[1] + 1) * (2 * r[2] + 1)
        # the entropy threshold's default kernel is the box of this job
        assert prm["te"] == oracle.entropy_te_default(st.hist, prm["w"], m)
        d = OFFSETS[ri % len(OFFSETS)]
        p = dict(prm, offset=d)
        cases = {
            MEAN: lambda x, y, z: b.mean(r, T, x, y, z),
            SIGMA: lambda x, y, z: b.sigma(r, 2, T, x, y, z),
            ENTROPY: lambda x, y, z: b.entropy(r, prm["te"], T, x, y, z),
            OKADA: lambda x, y, z: b.okada(r, prm["td"], T, x, y, z),
            OURS: lambda x, y, z: b.ours(r, d, T, x, y, z),
            OURS_CROSS7: lambda x, y, z: b.ours_layout("cross", r, d, T, x, y, z),
            OURS_CUBE: lambda x, y, z: b.ours_layout("cube", r, d, T, x, y, z),
            SIGMA_LOCAL: lambda x, y, z: b.sigma_local(r, 2, T, x, y, z),
        }
        for f, want in cases.items():
            got = oracle.filter_volume(vol, f, r, params=p)
            for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
                assert got[z, y, x] == want(x, y, z), (f, r, d, x, y, z)


@pytest.mark.parametrize("f", range(8))
def test_equal_axes_are_the_isotropic_filter(f):
    vol = phantoms.insect_phantom((14, 13, 12), 311, "u16")
    st = oracle.stats(vol)
    for r in (0, 1, 2):
        for d in (1, 2):
            iso = oracle.filter_volume(vol, f, r, params=dict(oracle.derive_params(st, r), offset=d))
            tri = oracle.filter_volume(vol, f, (r, r, r), params=dict(oracle.derive_params(st, (r, r, r)),
                                                                      offset=(d, d, d)))
            assert np.array_equal(iso, tri), (f, r, d)


@pytest.mark.parametrize("f", range(8))
def test_axis_permutation_symmetry(f):
    """Relabelling the axes of the volume and of the radii / offsets together
    relabels the output: F_{r o pi}(V o pi) = F_r(V) o pi for all six permutations."""
    vol = phantoms.random_volume((7, 6, 5), 321, "u16", vmax=4095)
    st = oracle.stats(vol)
    r, d = (2, 0, 1), (1, 2, 1)
    base = oracle.filter_volume(vol, f, r, params=dict(oracle.derive_params(st, r), offset=d))
    for perm in itertools.permutations(range(3)):
        # numpy axes are (z, y, x): volume axis a (x=0, y=1, z=2) is numpy axis 2 - a
        np_axes = [2 - perm[2 - i] for i in range(3)]
        pv = np.ascontiguousarray(np.transpose(vol, np_axes))
        pr = tuple(r[perm[a]] for a in range(3))
        pd = tuple(d[perm[a]] for a in range(3))
        got = oracle.filter_volume(pv, f, pr, params=dict(oracle.derive_params(st, pr), offset=pd))
        assert np.array_equal(got, np.transpose(base, np_axes)), (f, perm)


@pytest.mark.parametrize("r,d", [((2, 1, 0), (1, 1, 1)), ((0, 3, 1), (2, 1, 1)), ((1, 1, 2), (1, 2, 1))])
def test_spike_closed_forms(r, d):
    """A spike h on background b (gate off): the paper's filter keeps 3 of the
    9 (Mx + My + Mz) samples at the spike, A = b + (h - b) / (3 (Mx + My + Mz)),
    because the diagonal clusters' lines all miss the centre (every d_a >= 1);
    the mean gives b + (h - b) / (Mx My Mz)."""
    b, h = 100, 4000
    vol = np.full((15, 15, 15), b, np.uint16)
    vol[7, 7, 7] = h
    st = oracle.stats(vol)
    prm = dict(oracle.derive_params(st, r, oracle.Config(threshold_mode="none")), offset=d)
    L = sum(2 * a + 1 for a in r)
    ours = oracle.filter_volume(vol, OURS, r, params=prm)
    assert ours[7, 7, 7] == math.floor(b + Fraction(h - b, 3 * L) + Fraction(1, 2))
    box = (2 * r[0] + 1) * (2 * r[1] + 1) * (2 * r[2] + 1)
    mean = oracle.filter_volume(vol, MEAN, r, params=prm)
    assert mean[7, 7, 7] == math.floor(b + Fraction(h - b, box) + Fraction(1, 2))


def test_constant_volume_unchanged():
    vol = np.full((6, 7, 8), 777, np.uint16)
    st = oracle.stats(vol)
    for f in (MEAN, SIGMA, OKADA, OURS, OURS_CROSS7, OURS_CUBE, SIGMA_LOCAL):
        got = oracle.filter_volume(vol, f, (2, 0, 1), params=dict(oracle.derive_params(st, (2, 0, 1)),
                                                                    offset=(1, 2, 1)))
        assert (got == 777).all(), f


def test_spacing_radii():
    # round half up of extent / spacing, per axis
    assert oracle.spacing_radii(2.0, (1.0, 1.0, 2.5)) == (2, 2, 1)
    assert oracle.spacing_radii(1.5, (1.0, 3.0, 0.5)) == (2, 1, 3)
    assert oracle.spacing_radii(0.4, (1.0, 1.0, 1.0)) == (0, 0, 0)
    assert oracle.spacing_radii(3.0, (2.0, 6.0, 1.0)) == (2, 1, 3)
    for bad in ((0.0, 1.0, 1.0), (1.0, -1.0, 1.0), (1.0, 1.0, float("nan"))):
        with pytest.raises(ValueError):
            oracle.spacing_radii(2.0, bad)
