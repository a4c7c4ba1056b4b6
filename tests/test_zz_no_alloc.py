"""lnf_entropy_noalloc, the entry point for callers that cannot allocate
device memory (no context, no cudaMalloc): its result must equal the oracle's
image entropy and the ordinary lnf_entropy call's, on two calls in a row (the
shared scratch array keeps the previous call's counts and must be cleared each
time), with the dtype changing between calls.  This file is collected last on
purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_03119_gb300 as L
    from paper_1807_03119_gb300 import builder
    builder.build()
    lib = L.load()
    fn = lib.lnf_entropy_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return L, fn


def _dims(vol):
    nz, ny, nx = vol.shape
    return (ctypes.c_int64 * 3)(nx, ny, nz)


def test_noalloc_entropy_matches_oracle_and_lnf_entropy(lib):
    L, fn = lib
    # the dtype changes from call to call (u16 first, then u8, then u16 again)
    vols = [phantoms.insect_phantom((72, 40, 33), 5, "u16"), phantoms.P1(),
            phantoms.random_volume((31, 17, 9), 6, "u16"), phantoms.random_volume((5, 3, 2), 7, "u8")]
    stream = torch.cuda.current_stream()
    with L.Context() as ctx:
        for vol in vols:
            want = oracle.image_entropy(oracle.histogram(vol))   # the definition, on the host
            t = torch.from_numpy(vol).cuda()
            ref = ctx.entropy(t)           # the existing entry point
            assert abs(ref - want) <= 1e-9 * max(1.0, abs(want)), (ref, want)
            dH = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            for call in range(2):          # two calls in a row reuse the scratch array
                rc = fn(t.data_ptr(), _dims(vol), 0 if vol.dtype == np.uint8 else 1, dH.data_ptr(),
                        stream.cuda_stream)
                assert rc == 0
                torch.cuda.synchronize()
                got = float(dH.item())
                assert abs(got - want) <= 1e-9 * max(1.0, abs(want)), (call, got, want)
                assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (call, got, ref)


def test_noalloc_rejects_too_many_voxels(lib):
    _, fn = lib
    t = torch.zeros(8, dtype=torch.uint8, device="cuda")
    dH = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = (ctypes.c_int64 * 3)(1 << 16, 1 << 16, 1)      # 2^32 voxels: beyond the 32-bit counters
    assert fn(t.data_ptr(), big, 0, dH.data_ptr(), None) == 1
    assert fn(t.data_ptr(), (ctypes.c_int64 * 3)(2, 2, 2), 7, dH.data_ptr(), None) == 1
    assert fn(None, (ctypes.c_int64 * 3)(2, 2, 2), 0, dH.data_ptr(), None) == 1
