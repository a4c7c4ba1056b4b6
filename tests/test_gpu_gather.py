"""The gather kernels (whole volumes where few voxels pass the gate; every
other output is 0 by the gate's definition): bit-exact with the oracle and with
the plane-ring kernels (LNF_NO_GATHER) for all five filters at radius 1 and 2,
both dtypes, on volumes whose passing voxels include ones at the border (the
clamped taps), with the gate and threshold settings varied; dense volumes leave
the work to the ring kernels."""
import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FILTERS = [oracle.MEAN, oracle.SIGMA, oracle.ENTROPY, oracle.OKADA, oracle.OURS]


@pytest.fixture(scope="module")
def lnf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_03119_gb300 as L
    from paper_1807_03119_gb300 import builder
    builder.build()
    L.load()
    return L


def _sparse_u8(dims, seed):
    """Background noise around 20, a small bright ellipsoid, 0.1% salt, and
    bright voxels on the faces, edges and corners of the volume."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    v = np.clip(np.rint(rng.normal(20, 4, (nz, ny, nx))), 0, 255)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    v[((x - nx / 3) / 3) ** 2 + ((y - ny / 2) / 2) ** 2 + ((z - nz / 2) / 2) ** 2 <= 1] = 200
    salt = rng.random(v.shape) < 0.001
    v[salt] = 255
    v[0, 0, 0] = v[-1, -1, -1] = v[0, -1, 5] = v[3, 0, -1] = 240
    return v.astype(np.uint8)


def _sparse_u16(dims, seed):
    """12-bit background noise around 400, a small ellipsoid at 3000, 0.1% salt
    (4095), and bright voxels on the volume's faces."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    v = np.clip(np.rint(rng.normal(400, 30, (nz, ny, nx))), 0, 4095)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    v[((x - nx / 2) / 3) ** 2 + ((y - ny / 3) / 2) ** 2 + ((z - nz / 2) / 2) ** 2 <= 1] = 3000
    u = rng.random(v.shape)
    v[u < 0.001] = 4095
    v[0, 0, :8] = 4000
    v[-1, 3, -1] = v[5, -1, 0] = 3900
    return v.astype(np.uint16)


def _contexts(lnf, monkeypatch, **kw):
    with_g = lnf.Context(**kw)
    monkeypatch.setenv("LNF_NO_GATHER", "1")
    try:
        without = lnf.Context(**kw)
    finally:
        monkeypatch.delenv("LNF_NO_GATHER")
    return with_g, without


@pytest.mark.parametrize("dt,dims,seed", [("u16", (96, 40, 36), 701), ("u8", (128, 33, 29), 702),
                                          ("u16", (64, 64, 64), 703)])
@pytest.mark.parametrize("cfg", [{}, {"entropy_te": -1}, {"okada_td": 40}, {"threshold_mode": 1}])
def test_gather_matches_oracle_and_ring(lnf, monkeypatch, dt, dims, seed, cfg):
    vol = _sparse_u16(dims, seed) if dt == "u16" else _sparse_u8(dims, seed)
    st = oracle.stats(vol)
    ocfg = oracle.Config(okada_td=cfg.get("okada_td"), entropy_te=cfg.get("entropy_te"))
    kw = dict(cfg)
    if cfg.get("threshold_mode") == 1:   # a fixed threshold near the top: fewer voxels pass
        thr = int(np.percentile(vol, 99.9))
        kw["threshold_value"] = thr
        ocfg = oracle.Config(threshold_mode="fixed", threshold_value=thr)
    a, b = _contexts(lnf, monkeypatch, **kw)
    try:
        t = torch.from_numpy(vol).cuda()
        for r in (1, 2):
            prm = oracle.derive_params(st, r, ocfg)
            # few enough voxels pass for the gather kernel of every filter
            assert np.count_nonzero(vol >= prm["T"]) * 256 <= vol.size, "volume not sparse enough"
            for f in FILTERS:
                want = oracle.filter_volume(vol, f, r, params=prm)
                got = a.filter_volume(t, f, r).cpu().numpy()
                ring = b.filter_volume(t, f, r).cpu().numpy()
                assert np.array_equal(got, want), (f, r, int((got != want).sum()))
                assert np.array_equal(ring, want), (f, r, "ring")
            outs, H = a.filter_multi(t, FILTERS, r)
            Hh = H.cpu().numpy()
            for i, f in enumerate(FILTERS):
                want = oracle.filter_volume(vol, f, r, params=prm)
                assert np.array_equal(outs[i].cpu().numpy(), want)
                hw = oracle.image_entropy(oracle.histogram(want))
                assert abs(Hh[i + 1] - hw) <= 1e-9 * max(1.0, hw), (f, Hh[i + 1], hw)
    finally:
        a.close()
        b.close()


def test_dense_volume_leaves_the_work_to_the_ring_kernels(lnf):
    # half of the voxels pass: the gather kernels return at once, the ring kernels write
    vol = phantoms.random_volume((64, 48, 40), 711, "u16")
    st = oracle.stats(vol)
    with lnf.Context() as c:
        t = torch.from_numpy(vol).cuda()
        for f in FILTERS:
            got = c.filter_volume(t, f, 2).cpu().numpy()
            assert np.array_equal(got, oracle.filter_volume(vol, f, 2, params=oracle.derive_params(st, 2)))


@pytest.mark.parametrize("dt", ["u16", "u8"])
def test_fused_multi_filter_pass(lnf, monkeypatch, dt):
    """The fused kernel of a multi-filter call (mean, sigma, entropy filter and
    Okada from one pass) on a volume where few voxels pass the gate overall but a
    bright cube packs more than a round's worth (1024) into some block steps:
    outputs and entropies against the oracle and against the ring kernels alone.
    The cube fills one whole 128 x 32 block tile (4096 voxels per step: four rounds)
    at the volume's left border."""
    rng = np.random.default_rng(721)
    nx, ny, nz = 256, 128, 40
    if dt == "u16":
        vol = np.clip(np.rint(rng.normal(400, 30, (nz, ny, nx))), 0, 4095)
        vol[10:18, 32:64, 0:128] = rng.integers(2500, 3500, (8, 32, 128))
        vol[rng.random(vol.shape) < 0.002] = 4095
    else:
        vol = np.clip(np.rint(rng.normal(20, 4, (nz, ny, nx))), 0, 255)
        vol[10:18, 32:64, 0:128] = rng.integers(150, 220, (8, 32, 128))
        vol[rng.random(vol.shape) < 0.002] = 255
    vol = vol.astype(np.uint16 if dt == "u16" else np.uint8)
    st = oracle.stats(vol)
    a = lnf.Context()
    monkeypatch.setenv("LNF_NO_FUSED", "1")
    try:
        b = lnf.Context()
    finally:
        monkeypatch.delenv("LNF_NO_FUSED")
    try:
        t = torch.from_numpy(vol).cuda()
        for r in (1, 2):
            prm = oracle.derive_params(st, r)
            frac = np.count_nonzero(vol >= prm["T"]) / vol.size
            assert 1 / 256 < frac <= 1 / 32, frac   # the fused kernel's range, not the gather kernel's
            outs, H = a.filter_multi(t, FILTERS, r)
            outs_b, H_b = b.filter_multi(t, FILTERS, r)
            Hh = H.cpu().numpy()
            for i, f in enumerate(FILTERS):
                want = oracle.filter_volume(vol, f, r, params=prm)
                got = outs[i].cpu().numpy()
                assert np.array_equal(got, want), (f, r, int((got != want).sum()))
                assert np.array_equal(outs_b[i].cpu().numpy(), want), (f, r, "ring")
                hw = oracle.image_entropy(oracle.histogram(want))
                assert abs(Hh[i + 1] - hw) <= 1e-9 * max(1.0, hw), (f, Hh[i + 1], hw)
            assert np.allclose(H.cpu().numpy(), H_b.cpu().numpy(), rtol=1e-12, atol=0)
    finally:
        a.close()
        b.close()


def test_fused_pass_only_for_the_four_once(lnf):
    """The fused pass runs only when mean, sigma, entropy filter and Okada are each
    asked for once; repeated or partial lists take the ring kernels, with the
    same results (sparse volume: the fused pass would otherwise work)."""
    vol = _sparse_u16((96, 40, 36), 731)
    st = oracle.stats(vol)
    prm = oracle.derive_params(st, 2)
    want = {f: oracle.filter_volume(vol, f, 2, params=prm) for f in FILTERS}
    t = torch.from_numpy(vol).cuda()
    with lnf.Context() as c:
        for ids in ([oracle.MEAN, oracle.MEAN, oracle.SIGMA, oracle.ENTROPY, oracle.OKADA],
                    [oracle.SIGMA, oracle.OKADA], [oracle.OURS, oracle.OKADA, oracle.MEAN],
                    [oracle.OKADA, oracle.ENTROPY, oracle.SIGMA, oracle.MEAN, oracle.OURS, oracle.SIGMA]):
            outs, H = c.filter_multi(t, ids, 2)
            Hh = H.cpu().numpy()
            for i, f in enumerate(ids):
                got = outs[i].cpu().numpy()
                assert np.array_equal(got, want[f]), (ids, i, f)
                hw = oracle.image_entropy(oracle.histogram(want[f]))
                assert abs(Hh[i + 1] - hw) <= 1e-9 * max(1.0, hw), (ids, i, f)
