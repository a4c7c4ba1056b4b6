"""Python binding of liblnf, the GB300 local noise filter library (arXiv 1807.03119).

Argument marshalling only: every step of the filter path runs in the CUDA
kernels behind the C ABI of ``include/lnf.h``.  PyTorch supplies device memory
and streams.  Importing this package never falls back to anything: if the
compiled library is missing, ``load()`` raises.

Volumes are torch tensors of dtype uint8 or uint16 and shape (nz, ny, nx)
(x fastest), on the current CUDA device.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "MEAN", "SIGMA", "ENTROPY", "OKADA", "OURS", "OURS_CROSS7", "OURS_CUBE", "SIGMA_LOCAL", "ENTROPY_LOCAL", "FILTERS", "THRESH_OTSU", "THRESH_FIXED", "THRESH_NONE",
    "TD_AUTO", "TE_AUTO", "TE_PASS_ALL", "LnfError", "load", "build", "Context", "Config", "Job", "Request",
    "Result", "Params", "spacing_radii",
]

MEAN, SIGMA, ENTROPY, OKADA, OURS = 0, 1, 2, 3, 4
OURS_CROSS7, OURS_CUBE = 5, 6   # cluster-layout variants of the paper's filter
SIGMA_LOCAL = 7                 # the sigma filter with the local sigma of its cube
ENTROPY_LOCAL = 8               # the entropy filter with the grey-level probabilities of its cube
FILTERS = {"mean": MEAN, "sigma": SIGMA, "entropy": ENTROPY, "okada": OKADA, "ours": OURS,
           "ours_cross": OURS_CROSS7, "ours_cube": OURS_CUBE, "sigma_local": SIGMA_LOCAL,
           "entropy_local": ENTROPY_LOCAL}
THRESH_OTSU, THRESH_FIXED, THRESH_NONE = 0, 1, 2
TD_AUTO, TE_AUTO, TE_PASS_ALL = -1, -2, -1
STATUS = {0: "LNF_OK", 1: "LNF_EINVAL", 2: "LNF_ENOMEM", 3: "LNF_EBUDGET", 4: "LNF_EPENDING",
          5: "LNF_ECUDA", 6: "LNF_ETIMEOUT", 7: "LNF_ENOTFOUND", 8: "LNF_ECANCELLED"}
OK, EPENDING = 0, 4

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblnf.so")
_lib = None
_lock = threading.Lock()


class LnfError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class Config(ctypes.Structure):
    _fields_ = [
        ("stream", ctypes.c_void_p),
        ("hbm_budget_bytes", ctypes.c_uint64),
        ("max_inflight", ctypes.c_int32),
        ("threshold_mode", ctypes.c_int32),
        ("threshold_value", ctypes.c_uint32),
        ("sigma_k", ctypes.c_int32),
        ("okada_td", ctypes.c_int64),
        ("entropy_te_q", ctypes.c_int64),
        ("cluster_offset", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("entropy_local_te_q", ctypes.c_int64),
    ]


class Params(ctypes.Structure):
    _fields_ = [
        ("n_voxels", ctypes.c_uint64),
        ("sum", ctypes.c_uint64),
        ("sum_sq", ctypes.c_uint64),
        ("min_value", ctypes.c_uint32),
        ("max_value", ctypes.c_uint32),
        ("threshold", ctypes.c_uint32),
        ("sigma_band", ctypes.c_uint32),
        ("okada_td", ctypes.c_int64),
        ("weight_sum", ctypes.c_uint64),
        ("input_entropy", ctypes.c_double),
    ]


class Job(ctypes.Structure):
    _fields_ = [
        ("in_", ctypes.c_void_p),
        ("out", ctypes.c_void_p),
        ("dims", ctypes.c_int64 * 3),
        ("roi_origin", ctypes.c_int64 * 3),
        ("roi_dims", ctypes.c_int64 * 3),
        ("dtype", ctypes.c_int32),
        ("filter_id", ctypes.c_int32),
        ("radius", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("d_entropy", ctypes.c_void_p),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("vol_id", ctypes.c_int32),
        ("filter_id", ctypes.c_int32),
        ("radius", ctypes.c_int32),
        ("want_entropy", ctypes.c_int32),
        ("roi_origin", ctypes.c_int64 * 3),
        ("roi_dims", ctypes.c_int64 * 3),
        ("out_host", ctypes.c_void_p),
        ("arrival_time", ctypes.c_double),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("entropy", ctypes.c_double),
        ("t_admit", ctypes.c_double),
        ("t_start", ctypes.c_double),
        ("t_finish", ctypes.c_double),
    ]


class KernelTime(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 24),
        ("launches", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("total_ms", ctypes.c_double),
    ]


_i64p = ctypes.POINTER(ctypes.c_int64)
_SIGS = {
    "lnf_config_default": (None, [ctypes.POINTER(Config)]),
    "lnf_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "lnf_destroy": (None, [ctypes.c_void_p]),
    "lnf_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "lnf_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "lnf_version": (ctypes.c_char_p, []),
    "lnf_now": (ctypes.c_double, []),
    "lnf_filter_volume": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_void_p, _i64p, ctypes.c_int]),
    "lnf_filter_multi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, _i64p, ctypes.c_int,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "lnf_filter_multi_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, _i64p,
                                             ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.POINTER(ctypes.c_double)]),
    "lnf_filter_volume_aniso": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_void_p,
                                               _i64p, ctypes.c_int]),
    "lnf_filter_volume_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_void_p,
                                             _i64p]),
    "lnf_spacing_radii": (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int)]),
    "lnf_filter_roi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, _i64p,
                                      ctypes.c_int, _i64p, _i64p, ctypes.c_void_p]),
    "lnf_render": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, _i64p, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "lnf_selftest_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "lnf_entropy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _i64p, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double)]),
    "lnf_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Params), ctypes.c_void_p]),
    "lnf_debug_checks": (ctypes.c_int, []),
    "lnf_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "lnf_debug_poll": (ctypes.c_int, [ctypes.c_void_p]),
    "lnf_filter_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Job), ctypes.c_int]),
    "lnf_volume_register": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, _i64p,
                                           ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "lnf_volume_unregister": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lnf_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "lnf_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(Result)]),
    "lnf_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(Result)]),
    "lnf_result_copy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t]),
    "lnf_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "lnf_release": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "lnf_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lnf_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(KernelTime), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)]),
    "lnf_serving_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
}


def build(verbose=False, force=False):
    """Compile liblnf.so for sm_103a (nvcc; no GPU needed)."""
    from . import builder as _b
    return _b.build(verbose=verbose, force=force)


def load(path=None):
    """Load liblnf.so (or `path`, or the library the environment variable LNF_LIB
    names, e.g. the bounds-checking liblnf_debug.so) and declare its C
    signatures.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or os.environ.get("LNF_LIB") or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"liblnf.so not built at {p}: run paper_1807_03119_gb300.build() first")
            L = ctypes.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def spacing_radii(extent, spacing):
    """Per-axis radii (x, y, z), in voxels, of a physical extent on a grid of
    voxel spacing (sx, sy, sz): floor(extent / s_a + 1/2) (lnf_spacing_radii)."""
    L = load()
    out = (ctypes.c_int * 3)()
    sp = (ctypes.c_double * 3)(*[float(v) for v in spacing])
    rc = L.lnf_spacing_radii(float(extent), sp, out)
    if rc != OK:
        raise LnfError(rc, "lnf_spacing_radii: bad extent or spacing, or a radius above the maximum")
    return tuple(out)


def _dims_of(t):
    if t.dim() != 3:
        raise ValueError("volumes are 3-D tensors of shape (nz, ny, nx)")
    nz, ny, nx = t.shape
    return (ctypes.c_int64 * 3)(nx, ny, nz)


def _dtype_of(t):
    import torch
    if t.dtype == torch.uint8:
        return 0
    if t.dtype == torch.uint16:
        return 1
    raise TypeError("volumes are torch.uint8 or torch.uint16")


def _np_dtype_code(a):
    import numpy as np
    if a.dtype == np.uint8:
        return 0
    if a.dtype == np.uint16:
        return 1
    raise TypeError("volumes are uint8 or uint16")


def _check_dev(t):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("volume tensors must be contiguous CUDA tensors")


class Context:
    """One lnf_ctx.  Calls enqueue on torch's current stream at call time."""

    def __init__(self, threshold_mode=THRESH_OTSU, threshold_value=0, sigma_k=2, okada_td=TD_AUTO,
                 entropy_te=TE_AUTO, cluster_offset=1, autotune=False, hbm_budget_bytes=0,
                 max_inflight=0, stream=None, entropy_local_te=TE_AUTO):
        self.lib = load()
        cfg = Config()
        self.lib.lnf_config_default(ctypes.byref(cfg))
        cfg.threshold_mode = threshold_mode
        cfg.threshold_value = threshold_value
        cfg.sigma_k = sigma_k
        cfg.okada_td = okada_td
        cfg.entropy_te_q = entropy_te
        cfg.cluster_offset = cluster_offset
        cfg.entropy_local_te_q = entropy_local_te
        cfg.autotune = 1 if autotune else 0
        if hbm_budget_bytes:
            cfg.hbm_budget_bytes = hbm_budget_bytes
        if max_inflight:
            cfg.max_inflight = max_inflight
        self._fixed_stream = stream
        cfg.stream = self._stream_handle()
        h = ctypes.c_void_p()
        rc = self.lib.lnf_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != OK:
            raise LnfError(rc, "lnf_create failed")
        self.h = h
        self._debug = bool(self.lib.lnf_debug_checks())

    # -- plumbing
    def _stream_handle(self):
        if self._fixed_stream is not None:
            return self._fixed_stream
        import torch
        return torch.cuda.current_stream().cuda_stream

    def _sync_stream(self):
        self.lib.lnf_set_stream(self.h, self._stream_handle())

    def _check(self, rc):
        if rc == OK and self._debug:
            # a bounds-checking build: wait for the call's kernels and report a failed check
            rc = self.lib.lnf_debug_poll(self.h)
        if rc != OK:
            raise LnfError(rc, (self.lib.lnf_last_error(self.h) or b"").decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.lnf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- plain path
    def filter_volume(self, vol, filter_id, radius, out=None):
        import torch
        _check_dev(vol)
        if out is None:
            out = torch.empty_like(vol)
        self._sync_stream()
        self._check(self.lib.lnf_filter_volume(self.h, filter_id, radius, vol.data_ptr(), out.data_ptr(),
                                               _dims_of(vol), _dtype_of(vol)))
        return out

    def filter_volume_aniso(self, vol, filter_id, radius, offset=None, out=None):
        """Anisotropic voxel spacing: `radius` and `offset` (None: the context's
        cluster offset) are per-axis (x, y, z) triples."""
        import torch
        _check_dev(vol)
        if out is None:
            out = torch.empty_like(vol)
        rad = (ctypes.c_int * 3)(*[int(r) for r in radius])
        off = (ctypes.c_int * 3)(*[int(d) for d in offset]) if offset is not None else None
        self._sync_stream()
        self._check(self.lib.lnf_filter_volume_aniso(self.h, filter_id, rad, off, vol.data_ptr(), out.data_ptr(),
                                                     _dims_of(vol), _dtype_of(vol)))
        return out

    def filter_volume_f32(self, vol, filter_id, radius, offset=None, out=None):
        """A float32 volume, filtered on 65536 levels spanning its range
        (lnf_filter_volume_f32); `radius` is r or a per-axis (x, y, z) triple."""
        import torch
        _check_dev(vol)
        if vol.dtype != torch.float32:
            raise TypeError("filter_volume_f32 takes a float32 volume")
        if out is None:
            out = torch.empty_like(vol)
        r3 = tuple(radius) if isinstance(radius, (tuple, list)) else (radius,) * 3
        rad = (ctypes.c_int * 3)(*[int(r) for r in r3])
        off = (ctypes.c_int * 3)(*[int(d) for d in offset]) if offset is not None else None
        self._sync_stream()
        self._check(self.lib.lnf_filter_volume_f32(self.h, filter_id, rad, off, vol.data_ptr(), out.data_ptr(),
                                                   _dims_of(vol)))
        return out

    def filter_multi(self, vol, filter_ids, radius, outs=None, entropy=True, H=None):
        """All `filter_ids` at one radius; returns (outs, entropies tensor (n+1,) float64 or None).
        `H` may be a preallocated float64 CUDA tensor of n+1 entries."""
        import torch
        _check_dev(vol)
        n = len(filter_ids)
        if outs is None:
            outs = [torch.empty_like(vol) for _ in range(n)]
        ids = (ctypes.c_int * n)(*filter_ids)
        ptrs = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        if H is None and entropy:
            H = torch.zeros(n + 1, dtype=torch.float64, device=vol.device)
        self._sync_stream()
        self._check(self.lib.lnf_filter_multi(self.h, radius, vol.data_ptr(), _dims_of(vol), _dtype_of(vol), n,
                                              ids, ptrs, H.data_ptr() if H is not None else None))
        return outs, H

    def filter_multi_host(self, vol_np, filter_ids, radius, outs=None):
        """Host (numpy) buffers: copies in, filters, copies out; returns (outs, entropies list)."""
        import numpy as np
        n = len(filter_ids)
        nz, ny, nx = vol_np.shape
        dims = (ctypes.c_int64 * 3)(nx, ny, nz)
        if outs is None:
            outs = [np.empty_like(vol_np) for _ in range(n)]
        ids = (ctypes.c_int * n)(*filter_ids)
        ptrs = (ctypes.c_void_p * n)(*[o.ctypes.data for o in outs])
        H = (ctypes.c_double * (n + 1))()
        self._sync_stream()
        self._check(self.lib.lnf_filter_multi_host(self.h, radius, vol_np.ctypes.data, dims,
                                                   _np_dtype_code(vol_np), n, ids, ptrs, H))
        return outs, list(H)

    def filter_roi(self, vol, filter_id, radius, origin, size, out=None):
        """origin / size as (x, y, z); returns a tensor of shape (sz, sy, sx)."""
        import torch
        _check_dev(vol)
        if out is None:
            out = torch.empty((size[2], size[1], size[0]), dtype=vol.dtype, device=vol.device)
        self._sync_stream()
        self._check(self.lib.lnf_filter_roi(self.h, filter_id, radius, vol.data_ptr(), _dims_of(vol),
                                            _dtype_of(vol), (ctypes.c_int64 * 3)(*origin),
                                            (ctypes.c_int64 * 3)(*size), out.data_ptr()))
        return out

    def render(self, vol, filter_id, radius, view=4, with_depth=True, with_value=True):
        """Ray-cast the volume along `view` (0..5 = +x, -x, +y, -y, +z, -z) with
        the filter deciding at each candidate surface point; returns (image
        uint8, depth int32 or None, value int32 or None), each of shape (H, W)."""
        import torch
        _check_dev(vol)
        nz, ny, nx = vol.shape
        if view not in range(6):
            raise ValueError("view must be 0..5")
        H, W = {0: (nz, ny), 1: (nz, ny), 2: (nz, nx), 3: (nz, nx), 4: (ny, nx), 5: (ny, nx)}[view]
        image = torch.empty((H, W), dtype=torch.uint8, device=vol.device)
        depth = torch.empty((H, W), dtype=torch.int32, device=vol.device) if with_depth else None
        value = torch.empty((H, W), dtype=torch.int32, device=vol.device) if with_value else None
        self._sync_stream()
        self._check(self.lib.lnf_render(self.h, filter_id, radius, vol.data_ptr(), _dims_of(vol), _dtype_of(vol),
                                        view, image.data_ptr(), depth.data_ptr() if depth is not None else None,
                                        value.data_ptr() if value is not None else None))
        return image, depth, value

    def selftest_wait(self, limit_ms=50.0):
        """Failure-detection self-test: returns (status code, elapsed ms); the
        expected status is LNF_ETIMEOUT (6), the wait having given up."""
        el = ctypes.c_double()
        self._sync_stream()
        rc = self.lib.lnf_selftest_wait(self.h, limit_ms, ctypes.byref(el))
        return rc, el.value

    def entropy(self, vol):
        _check_dev(vol)
        H = ctypes.c_double()
        self._sync_stream()
        self._check(self.lib.lnf_entropy(self.h, vol.data_ptr(), _dims_of(vol), _dtype_of(vol), ctypes.byref(H)))
        return H.value

    def params(self, with_weights=False):
        """Parameters derived for the last analysed volume (dict), optionally the weight table."""
        import numpy as np
        p = Params()
        w = np.zeros(65536, np.uint32) if with_weights else None
        self._sync_stream()
        self._check(self.lib.lnf_get_params(self.h, ctypes.byref(p), w.ctypes.data if w is not None else None))
        d = {f: getattr(p, f) for f, _ in Params._fields_}
        if w is not None:
            d["weights"] = w   # 256 meaningful entries for uint8 volumes, 65536 for uint16
        return d

    # -- batched
    def filter_batch(self, jobs):
        """jobs: list of dicts with keys in, out, filter, radius, [roi_origin, roi_dims, entropy (tensor)]."""
        n = len(jobs)
        arr = (Job * n)()
        for i, j in enumerate(jobs):
            v = j["in"]
            _check_dev(v)
            _check_dev(j["out"])
            a = arr[i]
            a.in_ = v.data_ptr()
            a.out = j["out"].data_ptr()
            nz, ny, nx = v.shape
            a.dims[:] = [nx, ny, nz]
            if j.get("roi_dims"):
                a.roi_origin[:] = list(j["roi_origin"])
                a.roi_dims[:] = list(j["roi_dims"])
            a.dtype = _dtype_of(v)
            a.filter_id = j["filter"]
            a.radius = j["radius"]
            e = j.get("entropy")
            a.d_entropy = e.data_ptr() if e is not None else None
        self._sync_stream()
        self._check(self.lib.lnf_filter_batch(self.h, arr, n))

    # -- profiling
    def tuning(self):
        """The autotuner's choices: {"classes": [{dtype, filter, radius, zlen, ms}],
        "generic_zchunk": z chunk or 0}."""
        cap = 64
        cls = (ctypes.c_int32 * cap)()
        zl = (ctypes.c_int32 * cap)()
        ms = (ctypes.c_float * (4 * cap))()
        n = ctypes.c_int()
        gz = ctypes.c_int32()
        self._sync_stream()
        self._check(self.lib.lnf_get_tuning(self.h, cls, zl, ms, cap, ctypes.byref(n), ctypes.byref(gz)))
        out = []
        for k in range(min(n.value, cap)):
            c = cls[k]
            out.append({"dtype": "u8" if c // 256 == 0 else "u16", "filter": (c // 16) % 16, "radius": c % 16,
                        "zlen": zl[k], "ms": {z: ms[4 * k + q] for q, z in enumerate((4, 8, 16, 32))}})
        return {"classes": out, "generic_zchunk": gz.value}

    def profile(self, on=True):
        self._check(self.lib.lnf_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """({kind: (launches, total_ms)}, total kernel launches) since profile(True)."""
        arr = (KernelTime * 64)()
        n = ctypes.c_int()
        launches = ctypes.c_int64()
        self._check(self.lib.lnf_profile_read(self.h, arr, 64, ctypes.byref(n), ctypes.byref(launches)))
        return ({arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(min(n.value, 64))},
                launches.value)

    # -- serving
    def register_volume(self, vol):
        """Make a resident copy of a CUDA tensor or numpy array; returns its id."""
        import numpy as np
        vid = ctypes.c_int()
        self._sync_stream()
        if isinstance(vol, np.ndarray):
            vol = np.ascontiguousarray(vol)
            nz, ny, nx = vol.shape
            self._check(self.lib.lnf_volume_register(self.h, vol.ctypes.data, 1, (ctypes.c_int64 * 3)(nx, ny, nz),
                                                     _np_dtype_code(vol), ctypes.byref(vid)))
        else:
            _check_dev(vol)
            self._check(self.lib.lnf_volume_register(self.h, vol.data_ptr(), 0, _dims_of(vol), _dtype_of(vol),
                                                     ctypes.byref(vid)))
        return vid.value

    def unregister_volume(self, vid):
        self._check(self.lib.lnf_volume_unregister(self.h, vid))

    def submit(self, vol_id, filter_id, radius, out_host=None, roi_origin=None, roi_dims=None,
               want_entropy=False, arrival_time=0.0):
        r = Request()
        r.vol_id = vol_id
        r.filter_id = filter_id
        r.radius = radius
        r.want_entropy = 1 if want_entropy else 0
        if roi_dims is not None:
            r.roi_origin[:] = list(roi_origin)
            r.roi_dims[:] = list(roi_dims)
        r.out_host = out_host.ctypes.data if out_host is not None else None
        r.arrival_time = arrival_time
        t = ctypes.c_uint64()
        self._check(self.lib.lnf_submit(self.h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        res = Result()
        rc = self.lib.lnf_poll(self.h, ticket, ctypes.byref(res))
        if rc == EPENDING:
            return None
        self._check(rc)
        return res

    def wait(self, ticket, timeout_s=60.0):
        res = Result()
        self._check(self.lib.lnf_wait(self.h, ticket, timeout_s, ctypes.byref(res)))
        return res

    def result_copy(self, ticket, dst_np):
        self._check(self.lib.lnf_result_copy(self.h, ticket, dst_np.ctypes.data, dst_np.nbytes))
        return dst_np

    def cancel(self, ticket):
        return self.lib.lnf_cancel(self.h, ticket)

    def release(self, ticket):
        self._check(self.lib.lnf_release(self.h, ticket))

    def serving_stats(self):
        used = ctypes.c_uint64()
        q = ctypes.c_int()
        f = ctypes.c_int()
        self._check(self.lib.lnf_serving_stats(self.h, ctypes.byref(used), ctypes.byref(q), ctypes.byref(f)))
        return {"budget_used": used.value, "queued": q.value, "inflight": f.value}
