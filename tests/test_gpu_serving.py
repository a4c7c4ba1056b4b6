"""Serving (continuous batching) through the C ABI: results are the same
alone and in a concurrent mix, bit-exact with the oracle; admission honours
the HBM budget; queued requests can be cancelled; timings are ordered."""
import time

import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lnf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_03119_gb300 as L
    from paper_1807_03119_gb300 import builder
    builder.build()
    L.load()
    return L


def _vols():
    return [phantoms.insect_phantom((40, 36, 30), 2001, "u16"),
            phantoms.ellipsoid_phantom((33, 47, 21), 2002, "u8"),
            phantoms.insect_phantom((64, 32, 48), 2003, "u16")]


def _want(vol, f, r, roi=None):
    st = oracle.stats(vol)
    return oracle.filter_volume(vol, f, r, params=oracle.derive_params(st, r), roi=roi)


def _roi_shape(roi, vol):
    if roi is None:
        return vol.shape
    return (roi[5], roi[4], roi[3])


def test_alone_and_in_the_mix(lnf):
    vols = _vols()
    rng = np.random.default_rng(7)
    with lnf.Context() as c:
        ids = [c.register_volume(v) for v in vols]
        # the probe request, alone
        probe = (0, oracle.OURS, 2, (3, 4, 5, 20, 17, 11))
        v = vols[probe[0]]
        out_alone = np.zeros(_roi_shape(probe[3], v), v.dtype)
        tk = c.submit(ids[probe[0]], probe[1], probe[2], out_host=out_alone, roi_origin=probe[3][:3],
                      roi_dims=probe[3][3:], want_entropy=True, arrival_time=c.lib.lnf_now())
        res = c.wait(tk)
        assert res.status == 0
        want = _want(v, probe[1], probe[2], probe[3])
        assert np.array_equal(out_alone, want)
        assert abs(res.entropy - oracle.image_entropy(oracle.histogram(want))) <= 1e-9 * max(1, res.entropy)
        c.release(tk)
        # the same request submitted in the middle of a burst of 40 others
        reqs = []
        for k in range(41):
            if k == 20:
                vi, f, r, roi = probe
            else:
                vi = int(rng.integers(0, 3))
                f = int(rng.integers(0, 5))
                r = int(rng.integers(1, 4))
                vv = vols[vi]
                nz, ny, nx = vv.shape
                roi = None
                if rng.random() < 0.5:
                    bx, by, bz = (int(rng.integers(1, n + 1)) for n in (nx, ny, nz))
                    roi = (int(rng.integers(0, nx - bx + 1)), int(rng.integers(0, ny - by + 1)),
                           int(rng.integers(0, nz - bz + 1)), bx, by, bz)
            vv = vols[vi]
            out = np.zeros(_roi_shape(roi, vv), vv.dtype)
            tk = c.submit(ids[vi], f, r, out_host=out, roi_origin=roi[:3] if roi else None,
                          roi_dims=roi[3:] if roi else None, want_entropy=True, arrival_time=c.lib.lnf_now())
            reqs.append((tk, vi, f, r, roi, out))
        for tk, vi, f, r, roi, out in reqs:
            res = c.wait(tk)
            assert res.status == 0
            assert res.t_admit - 1e-3 <= res.t_start <= res.t_finish + 1e-6
            want = _want(vols[vi], f, r, roi)
            assert np.array_equal(out, want), (vi, f, r, roi)
            assert abs(res.entropy - oracle.image_entropy(oracle.histogram(want))) <= 1e-9 * max(1, res.entropy)
            c.release(tk)
        assert np.array_equal(reqs[20][5], out_alone)
        st = c.serving_stats()
        assert st["queued"] == 0 and st["inflight"] == 0


def _sparse_u16(dims, seed):
    """12-bit noise around 400 with a small bright ellipsoid and 0.1% salt: few
    voxels pass the Otsu gate."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    v = np.clip(np.rint(rng.normal(400, 30, (nz, ny, nx))), 0, 4095)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    v[((x - nx / 2) / 4) ** 2 + ((y - ny / 3) / 3) ** 2 + ((z - nz / 2) / 3) ** 2 <= 1] = 3000
    v[rng.random(v.shape) < 0.001] = 4095
    return v.astype(np.uint16)


def test_sigma_wide_radius_requests(lnf):
    # sigma at r = 3 and 4: the tap kernel takes a request while few voxels pass
    # the gate, the generic kernel otherwise; whole volumes and ROIs of a sparse
    # and a dense volume against the oracle
    sparse = _sparse_u16((61, 40, 37), 2101)
    dense = phantoms.random_volume((45, 30, 26), 2102, "u16")
    st = oracle.stats(sparse)
    for r in (3, 4):
        prm = oracle.derive_params(st, r)
        assert np.count_nonzero(sparse >= prm["T"]) * 32 <= sparse.size, "volume not sparse enough"
    with lnf.Context() as c:
        ids = [c.register_volume(v) for v in (sparse, dense)]
        cases = []
        for vi, vol in enumerate((sparse, dense)):
            nz, ny, nx = vol.shape
            for r in (3, 4):
                for roi in (None, (3, 5, 2, nx - 9, ny // 2, nz - 6)):
                    out = np.zeros(_roi_shape(roi, vol), vol.dtype)
                    tk = c.submit(ids[vi], oracle.SIGMA, r, out_host=out, roi_origin=roi[:3] if roi else None,
                                  roi_dims=roi[3:] if roi else None)
                    cases.append((tk, out, vol, r, roi))
        for tk, out, vol, r, roi in cases:
            c.wait(tk)
            assert np.array_equal(out, _want(vol, oracle.SIGMA, r, roi)), (vol.dtype, r, roi)
            c.release(tk)


def test_device_result_copy(lnf):
    vol = _vols()[1]
    with lnf.Context() as c:
        vid = c.register_volume(torch.from_numpy(vol).cuda())
        tk = c.submit(vid, oracle.SIGMA, 1)
        c.wait(tk)
        dst = np.zeros_like(vol)
        c.result_copy(tk, dst)
        assert np.array_equal(dst, _want(vol, oracle.SIGMA, 1))
        c.release(tk)
        with pytest.raises(lnf.LnfError):
            c.release(tk)


def test_budget_admission(lnf):
    vol = _vols()[0]
    nbytes = vol.nbytes
    with lnf.Context(hbm_budget_bytes=nbytes * 3) as c:
        vid = c.register_volume(vol)
        with pytest.raises(lnf.LnfError) as e:
            c.register_volume(np.zeros((64, 64, 64), np.uint16))   # 512 KiB > remaining budget
        assert e.value.status == 3
        # outputs that fit one at a time are all served
        outs = [np.zeros_like(vol) for _ in range(6)]
        tks = [c.submit(vid, oracle.MEAN, 1, out_host=o) for o in outs]
        for tk in tks:
            assert c.wait(tk).status == 0
            c.release(tk)
        want = _want(vol, oracle.MEAN, 1)
        assert all(np.array_equal(o, want) for o in outs)
    with lnf.Context(hbm_budget_bytes=nbytes + nbytes // 2) as c:
        vid = c.register_volume(vol)
        with pytest.raises(lnf.LnfError) as e:
            c.submit(vid, oracle.MEAN, 1)   # output alone exceeds the remaining budget
        assert e.value.status == 3


def test_cancel_queued(lnf):
    vol = phantoms.insect_phantom((96, 96, 96), 2010, "u16")
    with lnf.Context(max_inflight=1) as c:
        vid = c.register_volume(vol)
        tks = [c.submit(vid, oracle.SIGMA, 3) for _ in range(6)]
        rc = c.cancel(tks[-1])
        res = c.wait(tks[-1])
        if rc == 0:
            assert res.status == 8
        for tk in tks[:-1]:
            assert c.wait(tk).status == 0
            c.release(tk)
        with pytest.raises(lnf.LnfError):
            c.unregister_volume(12345)
        c.release(tks[-1])
        c.unregister_volume(vid)
