"""Parity of the variants with the oracle, through the C ABI: the
cluster-layout variants of the paper's filter (axis-cross and cube clusters),
the sigma filter with the local sigma of its cube and the entropy filter with
the grey-level probabilities of its cube; whole volumes and ROIs, both dtypes,
radii 0..2, cluster offsets 1 and 2, k = 1..3 or four entropy thresholds, and
the ray caster."""
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


def _few_level_volume(dims, seed, levels):
    """A u8 volume of `levels` grey levels (duplicates inside every cube), with a
    bright block so that the noise gate passes a part of it."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    v = rng.integers(0, levels, (nz, ny, nx)) * (200 // levels) + 20
    v[nz // 3: 2 * nz // 3, :, nx // 2:] += 30
    return v.astype(np.uint8)


@pytest.mark.parametrize("theta", [None, 0, -1, int(3.2 * (1 << oracle.ENTROPY_W_BITS))])
def test_entropy_local_matches_oracle(lnf, theta):
    """The entropy filter with the cube's own grey-level probabilities (id 8):
    whole volumes and ROIs at r = 0..2 on both dtypes and on a volume of few
    levels, the default, zero, pass-all and a 3.2-bit threshold, and the ray
    caster, bit-exact with the oracle."""
    kw = {} if theta is None else {"entropy_local_te": theta}
    cfg = oracle.Config(entropy_local_te=theta)
    mixed = False
    with lnf.Context(**kw) as c:
        for vol in _vols() + [_few_level_volume((29, 17, 13), 63, 9)]:
            t = torch.from_numpy(vol).cuda()
            st = oracle.stats(vol)
            for r in (0, 1, 2):
                prm = oracle.derive_params(st, r, cfg)
                got = c.filter_volume(t, oracle.ENTROPY_LOCAL, r).cpu().numpy()
                want = oracle.filter_volume(vol, oracle.ENTROPY_LOCAL, r, params=prm)
                assert np.array_equal(got, want), (vol.dtype, r, theta, int((got != want).sum()))
                kept = np.count_nonzero(want)
                mixed |= 0 < kept < np.count_nonzero(vol >= prm["T"])
                roi = (4, 3, 2, 11, 9, 8)
                got = c.filter_roi(t, oracle.ENTROPY_LOCAL, r, roi[:3], roi[3:]).cpu().numpy()
                want = oracle.filter_volume(vol, oracle.ENTROPY_LOCAL, r, params=prm, roi=roi)
                assert np.array_equal(got, want), ("roi", vol.dtype, r, theta)
            im, dep, val = c.render(t, oracle.ENTROPY_LOCAL, 1, 4)
            wim, wd, wv = oracle.render(vol, oracle.ENTROPY_LOCAL, 1, 4, params=oracle.derive_params(st, 1, cfg))
            assert np.array_equal(dep.cpu().numpy(), wd) and np.array_equal(im.cpu().numpy(), wim), theta
            c.params()   # raises LNF_ETIMEOUT if a bounded device wait gave up
    if theta not in (0, -1):   # (0 keeps every cube that is not constant, -1 every cube)
        assert mixed, "every case kept all or none of the gated voxels"
