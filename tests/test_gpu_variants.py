"""Parity of the variants with the oracle, through the C ABI: the
cluster-layout variants of the paper's filter (axis-cross and cube clusters)
and the sigma filter with the local sigma of its cube; whole volumes and
ROIs, both dtypes, radii 0..2, cluster offsets 1 and 2 or k = 1..3, and the
ray caster."""
import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VARIANTS = [oracle.OURS_CROSS7, oracle.OURS_CUBE]


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
    return [phantoms.insect_phantom((40, 27, 23), 61, "u16"),
            phantoms.insect_phantom((33, 21, 19), 62, "u8", background=20, lo=40, hi=220, sigma=25.0, vmax=255)]


@pytest.mark.parametrize("d", [1, 2])
def test_variants_match_oracle(lnf, d):
    with lnf.Context(cluster_offset=d) as c:
        for vol in _vols():
            t = torch.from_numpy(vol).cuda()
            st = oracle.stats(vol)
            for r in (0, 1, 2):
                prm = dict(oracle.derive_params(st, r), offset=d)
                for f in VARIANTS:
                    got = c.filter_volume(t, f, r).cpu().numpy()
                    want = oracle.filter_volume(vol, f, r, params=prm)
                    assert np.array_equal(got, want), (vol.dtype, f, r, d)
                    roi = (3, 2, 4, 17, 9, 7)
                    got = c.filter_roi(t, f, r, roi[:3], roi[3:]).cpu().numpy()
                    want = oracle.filter_volume(vol, f, r, params=prm, roi=roi)
                    assert np.array_equal(got, want), ("roi", vol.dtype, f, r, d)
            c.params()   # raises LNF_ETIMEOUT if a bounded device wait gave up


def test_variants_render(lnf):
    with lnf.Context() as c:
        for vol in _vols():
            t = torch.from_numpy(vol).cuda()
            st = oracle.stats(vol)
            prm = oracle.derive_params(st, 1)
            for f in VARIANTS:
                for view in (0, 3, 4):
                    im, dep, val = c.render(t, f, 1, view)
                    wim, wd, wv = oracle.render(vol, f, 1, view, params=prm)
                    assert np.array_equal(dep.cpu().numpy(), wd), (f, view)
                    assert np.array_equal(val.cpu().numpy().astype(np.uint32), wv), (f, view)
                    assert np.array_equal(im.cpu().numpy(), wim), (f, view)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sigma_local_matches_oracle(lnf, k):
    with lnf.Context(sigma_k=k) as c:
        for vol in _vols():
            t = torch.from_numpy(vol).cuda()
            st = oracle.stats(vol)
            for r in (0, 1, 2):
                prm = dict(oracle.derive_params(st, r, oracle.Config(sigma_k=k)), k=k)
                got = c.filter_volume(t, oracle.SIGMA_LOCAL, r).cpu().numpy()
                want = oracle.filter_volume(vol, oracle.SIGMA_LOCAL, r, params=prm)
                assert np.array_equal(got, want), (vol.dtype, r, k)
                roi = (5, 1, 2, 13, 11, 9)
                got = c.filter_roi(t, oracle.SIGMA_LOCAL, r, roi[:3], roi[3:]).cpu().numpy()
                want = oracle.filter_volume(vol, oracle.SIGMA_LOCAL, r, params=prm, roi=roi)
                assert np.array_equal(got, want), ("roi", vol.dtype, r, k)
            im, dep, val = c.render(t, oracle.SIGMA_LOCAL, 1, 4)
            prm = dict(oracle.derive_params(st, 1, oracle.Config(sigma_k=k)), k=k)
            wim, wd, wv = oracle.render(vol, oracle.SIGMA_LOCAL, 1, 4, params=prm)
            assert np.array_equal(dep.cpu().numpy(), wd) and np.array_equal(im.cpu().numpy(), wim)
            c.params()
