"""Pins of the oracle's ray caster (the paper's use of its filter: first
candidate surface point that the filter keeps, Sobel normal, Phong shading),
checked against geometry and closed forms rather than against its own code.

Shading constants and readings are stated in oracle/lnf_oracle.c; the closed
forms below follow from them: a surface facing the ray gives 255, a surface
seen edge-on gives round(255 * 0.1) = 26, and the Sobel operator answers a
linear field a*x + b*z exactly with g = (32a, 0, 32b) away from the borders.
"""
import math

import numpy as np
import pytest

import oracle

IDENT = 0      # mean at radius 0 is the identity (with the gate)
OURS = 4


def fixed(T):
    return oracle.Config(threshold_mode="fixed", threshold_value=T)


def test_facing_slab():
    nz, ny, nx = 24, 9, 11
    vol = np.zeros((nz, ny, nx), np.uint16)
    vol[7:] = 900
    im, d, val = oracle.render(vol, IDENT, 0, 4, cfg=fixed(500))
    assert (d == 7).all() and (im == 255).all() and (val == 900).all()
    # from the back the first sample is inside the slab; clamping at the face
    # leaves no gradient there, and g = 0 shades as facing
    im, d, val = oracle.render(vol, IDENT, 0, 5, cfg=fixed(500))
    assert (d == 0).all() and (im == 255).all()


def test_edge_on_face_and_misses():
    nz, ny, nx = 6, 5, 16
    vol = np.zeros((nz, ny, nx), np.uint8)
    vol[:, :, 9:] = 200                       # half space x >= 9, seen along +z
    im, d, _ = oracle.render(vol, IDENT, 0, 4, cfg=fixed(100))
    assert (d[:, :9] == -1).all() and (im[:, :9] == 0).all()
    assert (d[:, 9:] == 0).all()
    assert (im[:, 9] == 26).all()             # gradient along x only: c = 0
    assert (im[:, 10:] == 255).all()          # no gradient inside


@pytest.mark.parametrize("a,b,want", [(3, 4, 168), (1, 7, 229)])
def test_linear_ramp_shading(a, b, want):
    # P = a x + b z + 10: the first candidate along +z is interior, where the
    # Sobel gradient is (32a, 0, 32b) and c = b / sqrt(a^2 + b^2)
    nz, ny, nx = 40, 6, 12
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    vol = (a * x + b * z + 10).astype(np.uint16)
    T = 130
    im, d, _ = oracle.render(vol, IDENT, 0, 4, cfg=fixed(T))
    for xx in range(1, nx - 1):
        z0 = math.ceil((T - 10 - a * xx) / b)
        assert 1 <= z0 <= nz - 2
        assert (d[:, xx] == z0).all()
        assert (im[1:-1, xx] == want).all(), (xx, im[:, xx])


def test_sphere_depth_by_geometry():
    n = 21
    c, rho = (10, 9, 11), 6.5
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    inside = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= rho ** 2
    vol = np.where(inside, 300, 0).astype(np.uint16)
    _, d, _ = oracle.render(vol, IDENT, 0, 4, cfg=fixed(300))
    for yy in range(n):
        for xx in range(n):
            hits = [zz for zz in range(n) if inside[zz, yy, xx]]
            assert d[yy, xx] == (hits[0] if hits else -1)


def test_filter_rejects_spot_noise():
    nz, ny, nx = 30, 12, 12
    vol = np.zeros((nz, ny, nx), np.uint16)
    vol[20:] = 200
    clean = vol.copy()
    vol[5, 6, 6] = 200                         # a lone salt voxel in front
    _, d_id, _ = oracle.render(vol, IDENT, 0, 4, cfg=fixed(200))
    assert d_id[6, 6] == 5                     # the identity stops at it
    im, d, val = oracle.render(vol, OURS, 1, 4, cfg=fixed(200))
    im0, d0, val0 = oracle.render(clean, OURS, 1, 4, cfg=fixed(200))
    # the paper's filter calls it noise: the ray goes on to the slab, where the
    # gate holds once all nine clusters lie inside it (z = 20 + r + d)
    assert d[6, 6] == d0[6, 6] == 22
    assert (im == im0).all() and (d == d0).all() and (val == val0).all()


@pytest.mark.parametrize("f,r", [(0, 1), (1, 1), (3, 2), (4, 1), (2, 1)])
def test_views_agree_with_flipped_and_transposed_volumes(f, r):
    rng = np.random.default_rng(5)
    vol = rng.integers(0, 256, size=(9, 8, 7)).astype(np.uint8)
    vol[3:6, 2:6, 2:5] = 230
    prm = oracle.derive_params(oracle.stats(vol), r)
    ref = oracle.render(vol, f, r, 4, params=prm)
    back = oracle.render(vol[::-1].copy(), f, r, 5, params=prm)
    for a, b in zip(ref, back):
        assert (a == b).all()
    # +x of vol == +z of the volume whose z axis is vol's x axis
    vx = oracle.render(vol, f, r, 0, params=prm)
    vt = oracle.render(np.ascontiguousarray(vol.transpose(2, 0, 1)), f, r, 4, params=prm)
    for a, b in zip(vx, vt):
        assert (a == b).all()
    # +y of vol == +z of the volume whose z axis is vol's y axis
    vy = oracle.render(vol, f, r, 2, params=prm)
    vt = oracle.render(np.ascontiguousarray(vol.transpose(1, 0, 2)), f, r, 4, params=prm)
    for a, b in zip(vy, vt):
        assert (a == b).all()
