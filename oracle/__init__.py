"""CPU oracle for the local noise filter of arXiv 1807.03119.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product library never loads
it, and it shares no code with the CUDA path (the two only share the seeded
input generators in ``phantoms.py``).

What lives where:
  * ``lnf_oracle.c`` -- the per-voxel filters by literal enumeration of every
    tap (mean Eq. 4, sigma Eq. 5, Okada Eq. 6, entropy Eq. 7, the paper's
    nine-cluster filter Eq. 2-3), and the grey-level statistics;
  * this module -- the scalar parameter derivations in exact Python integer
    arithmetic: the Otsu threshold (Eq. 1), the sigma band, the Okada
    difference threshold, the entropy-filter weights and threshold, the
    fixed-point table and threshold of the entropy filter with the cube's own
    grey-level probabilities ("Related Work"), and the image entropy measure
    the paper uses to compare filters (Fig. 4).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` except the paper's printed fly-data numbers (T=101,
the Fig. 4 entropies), which need a dataset that is not available: those are
"parity unpinned" and are never asserted.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

__all__ = [
    "build", "lib", "Config", "stats", "otsu_threshold", "sigma_band", "okada_td_default",
    "log2_fixed", "entropy_weights", "entropy_te_default", "derive_params", "filter_volume",
    "filter_points", "image_entropy", "histogram", "MEAN", "SIGMA", "ENTROPY", "OKADA", "OURS",
    "FILTER_NAMES", "LOG2_FRAC_BITS", "ENTROPY_W_BITS", "spacing_radii", "quantize_f32", "dequantize_f32",
    "filter_volume_f32", "local_entropy_table", "local_entropy_te_default", "ENTROPY_LOCAL",
]

MEAN, SIGMA, ENTROPY, OKADA, OURS = 0, 1, 2, 3, 4
# cluster-layout variants of the paper's filter: axis-cross clusters (the
# commented-out S_0 at r = 1) and cube clusters
OURS_CROSS7, OURS_CUBE = 5, 6
# the sigma filter with the local standard deviation of its cube (Lee's original form)
SIGMA_LOCAL = 7
# the entropy filter with the grey-level probabilities of its own cube
ENTROPY_LOCAL = 8
FILTER_NAMES = {MEAN: "mean", SIGMA: "sigma", ENTROPY: "entropy", OKADA: "okada", OURS: "ours"}

# fixed point of the entropy-filter criterion (a stated reading: the paper gives
# the criterion in real numbers only)
LOG2_FRAC_BITS = 40
ENTROPY_W_BITS = 22

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lnf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblnf_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the C oracle with gcc (plain -O2, no fused multiply-add contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("filter_id", ctypes.c_int32),
        ("radius", ctypes.c_int32),
        ("offset", ctypes.c_int32),
        ("threshold", ctypes.c_uint32),
        ("sigma_band", ctypes.c_uint32),
        ("okada_td", ctypes.c_int64),
        ("entropy_te", ctypes.c_int64),
        ("entropy_w", ctypes.POINTER(ctypes.c_uint32)),
        ("sigma_k", ctypes.c_int32),
        ("aniso", ctypes.c_int32),
        ("rad", ctypes.c_int32 * 3),
        ("off", ctypes.c_int32 * 3),
        ("entropy_lt", ctypes.POINTER(ctypes.c_uint64)),
        ("entropy_lte", ctypes.c_int64),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # a test may point the oracle at a deliberately broken build of it
            # (tests/test_oracle_mutants.py) to show that the pins catch slips
            so = os.environ.get("LNF_ORACLE_SO") or build()
            L = ctypes.CDLL(so)
            i64 = ctypes.c_int64
            vp = ctypes.c_void_p
            L.oracle_filter_box.argtypes = [vp, i64, i64, i64, ctypes.c_int, ctypes.POINTER(_Params), vp,
                                            i64, i64, i64, i64, i64, i64]
            L.oracle_filter_box.restype = ctypes.c_int
            L.oracle_filter_points.argtypes = [vp, i64, i64, i64, ctypes.c_int, ctypes.POINTER(_Params),
                                               vp, i64, vp]
            L.oracle_filter_points.restype = ctypes.c_int
            L.oracle_stats.argtypes = [vp, i64, ctypes.c_int, vp, vp, vp, vp, vp, vp]
            L.oracle_stats.restype = ctypes.c_int
            L.oracle_render.argtypes = [vp, i64, i64, i64, ctypes.c_int, ctypes.POINTER(_Params), ctypes.c_int,
                                        vp, vp, vp]
            L.oracle_render.restype = ctypes.c_int
            _lib = L
    return _lib


def _dtype_code(vol):
    if vol.dtype == np.uint8:
        return 0
    if vol.dtype == np.uint16:
        return 1
    raise TypeError("oracle volumes are uint8 or uint16")


def _dims(vol):
    nz, ny, nx = vol.shape
    return int(nx), int(ny), int(nz)


# --------------------------------------------------------------------------- stats

class Stats:
    """Histogram h[v], N, S = sum P, Q = sum P^2, min, max of a volume."""

    def __init__(self, hist, N, S, Q, minv, maxv):
        self.hist, self.N, self.S, self.Q, self.minv, self.maxv = hist, N, S, Q, minv, maxv

    @property
    def levels(self):
        return len(self.hist)


def stats(vol):
    vol = np.ascontiguousarray(vol)
    L = 256 if _dtype_code(vol) == 0 else 65536
    hist = np.zeros(L, np.uint64)
    S = ctypes.c_uint64()
    qlo = ctypes.c_uint64()
    qhi = ctypes.c_uint64()
    mn = ctypes.c_uint32()
    mx = ctypes.c_uint32()
    rc = lib().oracle_stats(vol.ctypes.data, vol.size, _dtype_code(vol), hist.ctypes.data,
                            ctypes.byref(S), ctypes.byref(qlo), ctypes.byref(qhi),
                            ctypes.byref(mn), ctypes.byref(mx))
    if rc != 0:
        raise ValueError("oracle_stats failed")
    return Stats(hist, int(vol.size), int(S.value), (int(qhi.value) << 64) | int(qlo.value),
                 int(mn.value), int(mx.value))


def histogram(vol):
    return stats(vol).hist


# --------------------------------------------------------------------------- Eq. 1

def otsu_threshold(hist):
    """Otsu threshold T (Eq. 1): the grey level that minimises the within-class
    variance sigma_w^2(T) = w0 sigma0^2 + w1 sigma1^2, with class 0 = {v < T}
    and class 1 = {v >= T} (T is the lower limit of the foreground range).

    For fixed N and Q = sum v^2 h[v], N sigma_w^2 = Q - (S0^2/n0 + S1^2/n1), so
    the minimiser is the maximiser of J = S0^2/n0 + S1^2/n1, compared here as
    exact fractions.  Only T with both classes non-empty is eligible; ties go
    to the smallest T; a single-level histogram gives T = that level.
    """
    h = [int(c) for c in hist]
    N = sum(h)
    S = sum(v * c for v, c in enumerate(h))
    n0 = 0
    s0 = 0
    best_t = None
    best_j = None
    for t in range(1, len(h)):
        n0 += h[t - 1]
        s0 += (t - 1) * h[t - 1]
        n1 = N - n0
        if n0 == 0 or n1 == 0:
            continue
        j = Fraction(s0 * s0, n0) + Fraction((S - s0) ** 2, n1)
        if best_j is None or j > best_j:
            best_j, best_t = j, t
    if best_t is None:
        nz = [v for v, c in enumerate(h) if c > 0]
        return nz[0] if nz else 0
    return best_t


# --------------------------------------------------------------------------- Eq. 5, Eq. 6

def sigma_band(N, S, Q, k=2):
    """delta such that |d| <= k*sigma  <=>  |d| <= delta for integer d, with the
    population variance sigma^2 = (N Q - S^2) / N^2 of the whole volume."""
    num = k * k * (N * Q - S * S)
    return math.isqrt(num // (N * N))


def okada_td_default(N, S, Q):
    """Default Okada difference threshold (a reading: the paper only says
    'predefined'): T_d = floor(sigma) + 1, so that |d| < T_d <=> |d| <= sigma."""
    return math.isqrt((N * Q - S * S) // (N * N)) + 1


# --------------------------------------------------------------------------- Eq. 7

def log2_fixed(x):
    """floor-ish binary logarithm of the integer x >= 1 in fixed point with
    LOG2_FRAC_BITS fractional bits, by the classical repeated-squaring method:
    normalise x = 2^k m with m in [1, 2) held with 62 fractional bits, then
    square m once per fractional bit; a square >= 2 yields a 1 bit and is
    halved.  Each square is truncated to 62 fractional bits."""
    if x < 1:
        raise ValueError("log2_fixed needs x >= 1")
    k = x.bit_length() - 1
    one = 1 << 62
    m = (x << (62 - k)) if k <= 62 else (x >> (k - 62))
    res = k << LOG2_FRAC_BITS
    for i in range(1, LOG2_FRAC_BITS + 1):
        m = (m * m) >> 62
        if m >= 2 * one:
            m >>= 1
            res |= 1 << (LOG2_FRAC_BITS - i)
    return res


def entropy_weights(hist):
    """Fixed-point per-grey-level entropy terms of the entropy filter (Eq. 7):
    w[v] = round(2^22 * (-p_v log2 p_v)) with p_v = h[v]/N the normalized
    frequency of grey level v, computed as
        floor((2^22 * h * (lg N - lg h) + N 2^(F-1)) / (N 2^F))
    with lg the fixed-point log2 above (F fractional bits); w = 0 where h = 0."""
    h = [int(c) for c in hist]
    N = sum(h)
    F = LOG2_FRAC_BITS
    lgN = log2_fixed(N)
    w = np.zeros(len(h), np.uint32)
    den = N << F
    for v, c in enumerate(h):
        if c == 0:
            continue
        num = (c * (lgN - log2_fixed(c)) << ENTROPY_W_BITS) + (N << (F - 1))
        w[v] = num // den
    return w


def entropy_te_default(hist, w, m):
    """Default entropy threshold (a reading: the paper gives no value): the
    expected criterion of a kernel of m voxels drawn from the global grey-level
    distribution, floor(m * sum_v h[v] w[v] / N)."""
    h = [int(c) for c in hist]
    N = sum(h)
    tot = sum(c * int(wv) for c, wv in zip(h, w))
    return (m * tot) // N


def local_entropy_table(m):
    """Fixed point of the local entropy filter (a reading: the paper states the
    kernel's entropy in real numbers only): t[c] = round(2^22 c log2 c) for
    c = 0..m, computed as floor((c lg c + 2^(F-23)) / 2^(F-22)) with lg the
    fixed-point log2 above (F fractional bits); t[0] = t[1] = 0.  With c_g the
    number of cube voxels at grey level g, the cube's first order entropy is
    H = log2 m - (1/m) sum_g c_g log2 c_g, and m 2^22 H is t[m] - sum_g t[c_g]."""
    F, W = LOG2_FRAC_BITS, ENTROPY_W_BITS
    t = np.zeros(m + 1, np.uint64)
    for c in range(2, m + 1):
        t[c] = (c * log2_fixed(c) + (1 << (F - W - 1))) >> (F - W)
    return t


_local_tables = {}


def _local_table(m):
    """local_entropy_table(m), kept per m (read-only)."""
    with _lock:
        t = _local_tables.get(m)
        if t is None:
            t = _local_tables[m] = local_entropy_table(m)
            t.flags.writeable = False
        return t


def local_entropy_te_default(t, m):
    """Default threshold theta of the local entropy filter, in 2^-22 bits (a
    reading: the paper gives no value): half the largest entropy a cube of m
    voxels can have, log2(m) / 2, as floor(t[m] / (2 m))."""
    return int(t[m]) // (2 * m)


# --------------------------------------------------------------------------- params

class Config:
    """Filter configuration.  threshold_mode: 'otsu' (default), 'fixed' or 'none'."""

    def __init__(self, threshold_mode="otsu", threshold_value=0, sigma_k=2, okada_td=None,
                 entropy_te=None, offset=1, entropy_local_te=None):
        self.threshold_mode = threshold_mode
        self.threshold_value = threshold_value
        self.sigma_k = sigma_k
        self.okada_td = okada_td        # None -> floor(sigma) + 1
        self.entropy_te = entropy_te    # None -> expectation; -1 -> pass-all
        self.offset = offset
        self.entropy_local_te = entropy_local_te   # None -> log2(m)/2; -1 -> pass-all


def _axes(v):
    """An isotropic radius / offset r as (r, r, r); a per-axis (x, y, z) triple as itself."""
    if isinstance(v, (tuple, list, np.ndarray)):
        t = tuple(int(a) for a in v)
        if len(t) != 3:
            raise ValueError("per-axis values are (x, y, z) triples")
        return t
    return (int(v),) * 3


def spacing_radii(extent, spacing):
    """Per-axis radii (in voxels) of a physical extent on a grid of voxel
    spacing (sx, sy, sz): floor(extent / s_a + 1/2), rounded half up in IEEE
    double (a reading: the paper's volumes are isotropic)."""
    out = []
    for s in spacing:
        s = float(s)
        if not (s > 0 and math.isfinite(s)):
            raise ValueError("spacing must be positive and finite")
        out.append(int(math.floor(float(extent) / s + 0.5)))
    return tuple(out)


def derive_params(st, radius, cfg=None):
    """All scalar parameters of the five filters for a volume with stats `st`.
    `radius` is r, or a per-axis (rx, ry, rz) for anisotropic voxel spacing
    (the entropy threshold's kernel then has (2rx+1)(2ry+1)(2rz+1) voxels)."""
    cfg = cfg or Config()
    if cfg.threshold_mode == "otsu":
        T = otsu_threshold(st.hist)
    elif cfg.threshold_mode == "fixed":
        T = int(cfg.threshold_value)
    elif cfg.threshold_mode == "none":
        T = 0
    else:
        raise ValueError(cfg.threshold_mode)
    rx, ry, rz = _axes(radius)
    m = (2 * rx + 1) * (2 * ry + 1) * (2 * rz + 1)
    delta = sigma_band(st.N, st.S, st.Q, cfg.sigma_k)
    td = okada_td_default(st.N, st.S, st.Q) if cfg.okada_td is None else int(cfg.okada_td)
    w = entropy_weights(st.hist)
    te = entropy_te_default(st.hist, w, m) if cfg.entropy_te is None else int(cfg.entropy_te)
    # the local entropy filter's threshold: None = the default of the cube the
    # filter runs with (local_entropy_te_default), else the configured value
    lte = None if cfg.entropy_local_te is None else int(cfg.entropy_local_te)
    return {"T": T, "delta": delta, "td": td, "w": w, "te": te, "offset": cfg.offset,
            "radius": radius, "k": int(cfg.sigma_k), "lte": lte}


def _cparams(filter_id, prm):
    p = _Params()
    p.filter_id = filter_id
    rad, off = prm["radius"], prm["offset"]
    if isinstance(rad, (tuple, list, np.ndarray)) or isinstance(off, (tuple, list, np.ndarray)):
        p.aniso = 1
        p.rad[:] = list(_axes(rad))
        p.off[:] = list(_axes(off))
        p.radius = max(p.rad)
        p.offset = max(p.off)
    else:
        p.radius = rad
        p.offset = off
    p.threshold = prm["T"]
    p.sigma_band = min(prm["delta"], 0xFFFFFFFF)
    p.okada_td = prm["td"]
    p.entropy_te = prm["te"]
    w = np.ascontiguousarray(prm["w"], dtype=np.uint32)
    p.entropy_w = w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    p.sigma_k = int(prm.get("k", 2))
    # the local entropy filter: the table and the default threshold of this
    # call's cube
    rx, ry, rz = _axes(prm["radius"])
    m = (2 * rx + 1) * (2 * ry + 1) * (2 * rz + 1)
    lt = _local_table(m)
    p.entropy_lt = lt.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    lte = prm.get("lte")
    p.entropy_lte = local_entropy_te_default(lt, m) if lte is None else int(lte)
    return p, (w, lt)


def filter_volume(vol, filter_id, radius, cfg=None, params=None, roi=None, st=None):
    """Filter the whole volume (or the ROI (x0, y0, z0, nx, ny, nz)); the halo
    always comes from the full volume and the statistics from the full volume.
    `radius` (and the cluster offset in `cfg` / `params`) may be a per-axis
    (x, y, z) triple for anisotropic voxel spacing."""
    vol = np.ascontiguousarray(vol)
    nx, ny, nz = _dims(vol)
    if params is None:
        params = derive_params(st or stats(vol), radius, cfg)
    else:
        params = dict(params, radius=radius)
    if roi is None:
        roi = (0, 0, 0, nx, ny, nz)
    x0, y0, z0, bx, by, bz = (int(v) for v in roi)
    out = np.zeros((bz, by, bx), vol.dtype)
    p, keep = _cparams(filter_id, params)
    rc = lib().oracle_filter_box(vol.ctypes.data, nx, ny, nz, _dtype_code(vol), ctypes.byref(p),
                                 out.ctypes.data, x0, x0 + bx, y0, y0 + by, z0, z0 + bz)
    del keep
    if rc != 0:
        raise ValueError("oracle_filter_box rejected its arguments")
    return out


def filter_points(vol, filter_id, radius, pts, params):
    """Filter values at the given (x, y, z) points (array of shape (n, 3))."""
    vol = np.ascontiguousarray(vol)
    nx, ny, nz = _dims(vol)
    pts = np.ascontiguousarray(pts, dtype=np.int64).reshape(-1, 3)
    vals = np.zeros(len(pts), np.uint32)
    p, keep = _cparams(filter_id, dict(params, radius=radius))
    rc = lib().oracle_filter_points(vol.ctypes.data, nx, ny, nz, _dtype_code(vol), ctypes.byref(p),
                                    pts.ctypes.data, len(pts), vals.ctypes.data)
    del keep
    if rc != 0:
        raise ValueError("oracle_filter_points rejected its arguments")
    return vals


# --------------------------------------------------------------------------- float32 volumes

def quantize_f32(vol):
    """The 65536 grey levels of a float32 volume (a reading: the paper filters
    grey levels): with lo / hi the volume's min / max and d = hi - lo, level
    q = floor((v - lo) * (65535 / d) + 1/2), every q = 0 when d = 0.  Each step
    is one IEEE float32 operation rounded to nearest, in this order.
    Returns (levels uint16, lo, hi)."""
    vol = np.ascontiguousarray(vol, dtype=np.float32)
    if not np.isfinite(vol).all():
        raise ValueError("float32 volumes must hold finite values")
    lo, hi = np.float32(vol.min()), np.float32(vol.max())
    d = np.float32(hi - lo)
    if not np.isfinite(d):
        raise ValueError("the range is wider than float32 holds")
    if d == 0:
        return np.zeros(vol.shape, np.uint16), lo, hi
    sc = np.float32(np.float32(65535.0) / d)
    t = (vol - lo) * sc + np.float32(0.5)
    assert t.dtype == np.float32
    return np.minimum(np.floor(t), np.float32(65535.0)).astype(np.uint16), lo, hi


def dequantize_f32(q, lo, hi):
    """value(q) = lo + q * (d / 65535) in float32 (one rounding per operation)."""
    lo, hi = np.float32(lo), np.float32(hi)
    step = np.float32(np.float32(hi - lo) / np.float32(65535.0))
    out = lo + q.astype(np.float32) * step
    assert out.dtype == np.float32
    return out


def filter_volume_f32(vol, filter_id, radius, cfg=None, offset=None):
    """A float32 volume: quantised to levels, filtered by the 16-bit oracle
    (statistics and parameters of the levels), mapped back to float32."""
    q, lo, hi = quantize_f32(vol)
    st = stats(q)
    prm = derive_params(st, radius, cfg)
    if offset is not None:
        prm = dict(prm, offset=offset)
    return dequantize_f32(filter_volume(q, filter_id, radius, params=prm), lo, hi)


def render_extent(shape, view):
    """(H, W) of the image rendered along view 0..5 (+x, -x, +y, -y, +z, -z)
    from a volume of numpy shape (nz, ny, nx)."""
    nz, ny, nx = shape
    return {0: (nz, ny), 1: (nz, ny), 2: (nz, nx), 3: (nz, nx), 4: (ny, nx), 5: (ny, nx)}[view]


def render(vol, filter_id, radius, view, params=None, cfg=None, st=None):
    """Ray-cast the volume along `view` with the filter deciding at each
    candidate surface point (the paper's use of its filter; readings in the C
    source): returns (image uint8, depth int32, value uint32), each (H, W)."""
    vol = np.ascontiguousarray(vol)
    nx, ny, nz = _dims(vol)
    if params is None:
        params = derive_params(st or stats(vol), radius, cfg)
    else:
        params = dict(params, radius=radius)
    H, W = render_extent(vol.shape, view)
    image = np.zeros((H, W), np.uint8)
    depth = np.zeros((H, W), np.int32)
    value = np.zeros((H, W), np.uint32)
    p, keep = _cparams(filter_id, params)
    rc = lib().oracle_render(vol.ctypes.data, nx, ny, nz, _dtype_code(vol), ctypes.byref(p), int(view),
                             image.ctypes.data, depth.ctypes.data, value.ctypes.data)
    del keep
    if rc != 0:
        raise ValueError("oracle_render rejected its arguments")
    return image, depth, value


# --------------------------------------------------------------------------- Fig. 4

def image_entropy(hist):
    """Shannon entropy H = -sum_v (c_v/N) log2(c_v/N) of a grey-level histogram
    (the measure of the paper's Fig. 4; lower is better), summed with fsum."""
    h = [int(c) for c in hist if int(c) > 0]
    N = sum(h)
    if N == 0:
        return 0.0
    return math.fsum(-(c / N) * math.log2(c / N) for c in h)
