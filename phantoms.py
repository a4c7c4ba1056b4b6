"""Seeded synthetic CT-like phantoms (input generators only).

The paper evaluates its filters on an SRµCT scan of a tachinid fly (§"CT Data and
3D Visualisation"), which is not available here.  These generators stand in for
it: grey-value volumes with thin shells, tubes, cavities and blobs on a dark
background, corrupted by Gaussian noise and (optionally) salt-and-pepper spots,
which is the kind of "spot noise" the paper's filter is meant to suppress.

This module holds NO filter arithmetic: it only draws inputs.  Both the CUDA
path's tests/benchmark and the CPU oracle's tests take their inputs from here.

Layout convention: a volume with dims (nx, ny, nz) is a C-ordered numpy array of
shape (nz, ny, nx), i.e. x is the fastest-varying index:
``idx = (z * ny + y) * nx + x``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "ellipsoid_phantom",
    "insect_phantom",
    "random_volume",
    "dtype_of",
    "P1",
    "P2",
    "P3",
    "batch_volume_specs",
]


def dtype_of(name):
    """numpy dtype for 'u8' / 'u16' (or an existing numpy dtype)."""
    if name in ("u8", "uint8", np.uint8):
        return np.uint8
    if name in ("u16", "uint16", np.uint16):
        return np.uint16
    raise ValueError(f"unsupported dtype {name!r}")


def _finish(vol_f, rng, sigma, salt_pepper, vmax, dtype):
    """Add Gaussian noise (round half to even), optional salt-and-pepper, clip."""
    if sigma > 0:
        noise = rng.standard_normal(vol_f.shape, dtype=np.float32)
        noise *= np.float32(sigma)
        vol_f += noise
        del noise
    np.rint(vol_f, out=vol_f)
    np.clip(vol_f, 0, vmax, out=vol_f)
    out = vol_f.astype(dtype)
    del vol_f
    if salt_pepper > 0:
        n = out.size
        k = int(round(n * salt_pepper))
        idx = rng.choice(n, size=k, replace=False) if n <= 1 << 22 else rng.integers(0, n, size=k)
        flat = out.reshape(-1)
        half = k // 2
        flat[idx[:half]] = vmax  # salt
        flat[idx[half:]] = 0  # pepper
    return out


def _grid(lo, hi):
    """Open grids (z, y, x) of voxel centres for a bounding box [lo, hi)."""
    z = np.arange(lo[2], hi[2], dtype=np.float32)[:, None, None]
    y = np.arange(lo[1], hi[1], dtype=np.float32)[None, :, None]
    x = np.arange(lo[0], hi[0], dtype=np.float32)[None, None, :]
    return x, y, z


def _random_rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array(
        [
            [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
            [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
            [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
        ],
        dtype=np.float32,
    )


def _paint_ellipsoid(vol, centre, axes, value, shell=None, rot=None):
    """Paint a (possibly rotated) ellipsoid or ellipsoidal shell of thickness `shell`."""
    nz, ny, nx = vol.shape
    ext = float(max(axes)) + 1.0
    lo = [max(0, int(np.floor(centre[i] - ext))) for i in range(3)]
    hi = [min((nx, ny, nz)[i], int(np.ceil(centre[i] + ext)) + 1) for i in range(3)]
    if any(h <= l for l, h in zip(lo, hi)):
        return
    x, y, z = _grid(lo, hi)
    dx, dy, dz = x - centre[0], y - centre[1], z - centre[2]
    if rot is not None:
        u = rot[0, 0] * dx + rot[0, 1] * dy + rot[0, 2] * dz
        v = rot[1, 0] * dx + rot[1, 1] * dy + rot[1, 2] * dz
        w = rot[2, 0] * dx + rot[2, 1] * dy + rot[2, 2] * dz
    else:
        u, v, w = dx, dy, dz
    f = (u / axes[0]) ** 2 + (v / axes[1]) ** 2 + (w / axes[2]) ** 2
    inside = f <= 1.0
    if shell is not None:
        a_min = float(min(axes))
        inner = max(0.0, 1.0 - shell / a_min)
        inside &= f >= inner * inner
    sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    sub[inside] = value


def _paint_tube(vol, p0, p1, radius, value):
    """Paint a capsule (segment p0-p1 with the given radius)."""
    nz, ny, nx = vol.shape
    p0 = np.asarray(p0, np.float32)
    p1 = np.asarray(p1, np.float32)
    lo = [max(0, int(np.floor(min(p0[i], p1[i]) - radius - 1))) for i in range(3)]
    hi = [min((nx, ny, nz)[i], int(np.ceil(max(p0[i], p1[i]) + radius + 1)) + 1) for i in range(3)]
    if any(h <= l for l, h in zip(lo, hi)):
        return
    x, y, z = _grid(lo, hi)
    d = p1 - p0
    dd = float(np.dot(d, d)) or 1.0
    t = ((x - p0[0]) * d[0] + (y - p0[1]) * d[1] + (z - p0[2]) * d[2]) / dd
    t = np.clip(t, 0.0, 1.0)
    ex = x - (p0[0] + t * d[0])
    ey = y - (p0[1] + t * d[1])
    ez = z - (p0[2] + t * d[2])
    inside = ex * ex + ey * ey + ez * ez <= radius * radius
    sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    sub[inside] = value


def ellipsoid_phantom(dims, seed, dtype="u8", n_objects=6, background=20, lo=40, hi=220,
                      sigma=20.0, salt_pepper=0.0, vmax=None):
    """Blobs and shells phantom: `n_objects` random ellipsoids / ellipsoidal shells
    (axis-aligned or randomly rotated, shell thickness 1-3 voxels) with intensities
    uniform in [lo, hi] on a constant background, plus Gaussian noise, clipped."""
    nx, ny, nz = (int(d) for d in dims)
    dt = dtype_of(dtype)
    if vmax is None:
        vmax = int(np.iinfo(dt).max)
    rng = np.random.default_rng(seed)
    vol = np.full((nz, ny, nx), float(background), dtype=np.float32)
    size = np.array([nx, ny, nz], np.float32)
    for _ in range(n_objects):
        centre = rng.uniform(0.2, 0.8, 3) * size
        axes = rng.uniform(0.08, 0.3, 3) * size.min()
        axes = np.maximum(axes, 2.0)
        value = float(rng.integers(lo, hi + 1))
        shell = float(rng.integers(1, 4)) if rng.random() < 0.5 else None
        rot = _random_rotation(rng) if rng.random() < 0.5 else None
        _paint_ellipsoid(vol, centre, axes, value, shell=shell, rot=rot)
    return _finish(vol, rng, sigma, salt_pepper, vmax, dt)


def insect_phantom(dims, seed, dtype="u16", background=400, lo=1200, hi=3600, sigma=150.0,
                   salt_pepper=0.01, vmax=4095, n_inner_shells=8, n_tubes=12, n_cavities=6):
    """Insect-like phantom: a thin body shell (1-3 voxels) around ~70% of the box,
    thin inner shells, tubes of radius 2-6 along random segments, cavities filled
    with background, Gaussian noise and salt-and-pepper spots (half to vmax, half to 0)."""
    nx, ny, nz = (int(d) for d in dims)
    dt = dtype_of(dtype)
    rng = np.random.default_rng(seed)
    vol = np.full((nz, ny, nx), float(background), dtype=np.float32)
    size = np.array([nx, ny, nz], np.float32)
    centre = size / 2.0
    scale = max(1.0, float(size.min()) / 512.0)
    body_axes = 0.35 * size * rng.uniform(0.9, 1.0, 3)
    _paint_ellipsoid(vol, centre, body_axes, float(rng.integers(lo, hi + 1)),
                     shell=float(rng.integers(1, 4)))
    for _ in range(n_inner_shells):
        c = centre + rng.uniform(-0.2, 0.2, 3) * size
        axes = rng.uniform(0.04, 0.15, 3) * size
        axes = np.maximum(axes, 3.0)
        _paint_ellipsoid(vol, c, axes, float(rng.integers(lo, hi + 1)),
                         shell=float(rng.integers(1, 4)),
                         rot=_random_rotation(rng) if rng.random() < 0.5 else None)
    for _ in range(n_tubes):
        p0 = centre + rng.uniform(-0.3, 0.3, 3) * size
        p1 = centre + rng.uniform(-0.3, 0.3, 3) * size
        radius = float(rng.uniform(2.0, 6.0)) * scale
        _paint_tube(vol, p0, p1, radius, float(rng.integers(lo, hi + 1)))
    for _ in range(n_cavities):
        c = centre + rng.uniform(-0.2, 0.2, 3) * size
        axes = rng.uniform(0.02, 0.06, 3) * size
        axes = np.maximum(axes, 2.0)
        _paint_ellipsoid(vol, c, axes, float(background))
    return _finish(vol, rng, sigma, salt_pepper, vmax, dt)


def random_volume(dims, seed, dtype="u8", vmin=0, vmax=None, p_extreme=0.1):
    """Uniform random grey values in [vmin, vmax]; a fraction `p_extreme` of voxels
    is forced to vmin or vmax so that both extremes are always exercised."""
    nx, ny, nz = (int(d) for d in dims)
    dt = dtype_of(dtype)
    if vmax is None:
        vmax = int(np.iinfo(dt).max)
    rng = np.random.default_rng(seed)
    vol = rng.integers(vmin, vmax + 1, size=(nz, ny, nx), dtype=np.int64)
    if p_extreme > 0:
        m = rng.random(vol.shape) < p_extreme
        ext = np.where(rng.random(vol.shape) < 0.5, vmin, vmax)
        vol[m] = ext[m]
    return vol.astype(dt)


# Named workloads ---------------------------------------------------------------

def P1(seed=1):
    """64^3 uint8: 6 random ellipsoids/shells, intensities 40-220 on background 20,
    Gaussian sigma 20, clipped to [0, 255]."""
    return ellipsoid_phantom((64, 64, 64), seed, "u8", n_objects=6, background=20,
                             lo=40, hi=220, sigma=20.0)


def P2(seed=2, dims=(512, 512, 512)):
    """512^3 uint16, 12-bit insect-like phantom: background 400, structures
    1200-3600, Gaussian sigma 150, 1% salt-and-pepper, clipped to [0, 4095]."""
    return insect_phantom(dims, seed, "u16", background=400, lo=1200, hi=3600,
                          sigma=150.0, salt_pepper=0.01, vmax=4095)


def P3(seed=3, dims=(1024, 1024, 1024)):
    """1024^3 uint8: the insect-like generator rescaled to 8 bits (background 20,
    structures 40-220), Gaussian sigma 25, 1% salt-and-pepper, clipped to [0, 255]."""
    return insect_phantom(dims, seed, "u8", background=20, lo=40, hi=220,
                          sigma=25.0, salt_pepper=0.01, vmax=255)


def batch_volume_specs(n=64, seed=1000, lo=96, hi=384):
    """Specs of the uneven batch: each dim uniform in [lo, hi] independently
    (non-cubic), even index uint8 (blob phantom), odd index uint16 (insect
    phantom), radius uniform in {1, 2}.  Returns a list of dicts."""
    specs = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        dims = tuple(int(v) for v in rng.integers(lo, hi + 1, size=3))
        radius = int(rng.integers(1, 3))
        specs.append({"index": i, "dims": dims, "dtype": "u8" if i % 2 == 0 else "u16",
                      "radius": radius, "seed": seed + i})
    return specs


def batch_volume(spec):
    """Generate the volume for one entry of `batch_volume_specs`."""
    if spec["dtype"] == "u8":
        return ellipsoid_phantom(spec["dims"], spec["seed"], "u8", n_objects=6,
                                 background=20, lo=40, hi=220, sigma=20.0)
    return insect_phantom(spec["dims"], spec["seed"], "u16", background=400, lo=1200,
                          hi=3600, sigma=150.0, salt_pepper=0.01, vmax=4095)
