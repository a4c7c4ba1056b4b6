"""The gate-first kernel (whole volumes while few voxels pass the noise gate;
every other output is 0 by the gate's definition, Eq. 6 / Eq. 7 "0,
otherwise"): bit-exact with the oracle and with the plane-ring kernels
(LNF_NO_GATE) for all five filters at radius 1..4, both dtypes, single-filter
and five-filter calls with their output entropies, on volumes whose passing
voxels include ones on the faces, edges and corners (the clamped taps), with
odd widths and voxel counts that are not a multiple of 8 or of a bitmask
chunk; regions where every voxel passes; repeated and partial filter lists;
dense volumes leave the work to the ring kernels."""
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
    v[rng.random(v.shape) < 0.001] = 255
    v[0, 0, 0] = v[-1, -1, -1] = v[0, -1, min(5, nx - 1)] = v[min(3, nz - 1), 0, -1] = 240
    return v.astype(np.uint8)


def _sparse_u16(dims, seed):
    """12-bit background noise around 400, a small ellipsoid at 3000, 0.1% salt
    (4095), and bright voxels on the volume's faces, edges and corners."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    v = np.clip(np.rint(rng.normal(400, 30, (nz, ny, nx))), 0, 4095)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    v[((x - nx / 2) / 3) ** 2 + ((y - ny / 3) / 2) ** 2 + ((z - nz / 2) / 2) ** 2 <= 1] = 3000
    v[rng.random(v.shape) < 0.001] = 4095
    v[0, 0, :8] = 4000
    v[-1, min(3, ny - 1), -1] = v[min(5, nz - 1), -1, 0] = 3900
    v[-1, -1, -1] = v[0, -1, -1] = 3800
    return v.astype(np.uint16)


def _tiny(dims, seed, dt):
    """A volume smaller than one tile and its halo: noise with three bright voxels
    (two corners and one face)."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    hi = 4095 if dt == "u16" else 255
    v = np.clip(np.rint(rng.normal(hi // 10, hi // 100, (nz, ny, nx))), 0, hi)
    v[0, 0, 0] = v[-1, -1, -1] = v[nz // 2, 0, nx // 2] = hi - 5
    return v.astype(np.uint16 if dt == "u16" else np.uint8)


def _ring_context(lnf, monkeypatch, **kw):
    monkeypatch.setenv("LNF_NO_GATE", "1")
    try:
        return lnf.Context(**kw)
    finally:
        monkeypatch.delenv("LNF_NO_GATE")


def _check_multi(ctx, t, vol, r, prm, ids=FILTERS, wants=None):
    outs, H = ctx.filter_multi(t, ids, r)
    Hh = H.cpu().numpy()
    for i, f in enumerate(ids):
        want = wants[f] if wants else oracle.filter_volume(vol, f, r, params=prm)
        got = outs[i].cpu().numpy()
        assert np.array_equal(got, want), (f, r, int((got != want).sum()))
        hw = oracle.image_entropy(oracle.histogram(want))
        assert abs(Hh[i + 1] - hw) <= 1e-9 * max(1.0, hw), (f, Hh[i + 1], hw)
    return outs, H


CASES = [("u16", (96, 40, 36), 701, (1, 2, 3, 4)), ("u8", (128, 33, 29), 702, (1, 2, 4)),
         ("u16", (64, 64, 64), 703, (2,)), ("u16", (93, 37, 21), 704, (1, 2)), ("u8", (37, 70, 19), 705, (2, 3)),
         ("u16", (9, 7, 4), 706, (1, 4))]


@pytest.mark.parametrize("dt,dims,seed,radii", CASES)
@pytest.mark.parametrize("cfg", [{}, {"entropy_te": -1}, {"okada_td": 40}, {"threshold_mode": 1}])
def test_gate_matches_oracle_and_ring(lnf, monkeypatch, dt, dims, seed, radii, cfg):
    if dims[0] * dims[1] * dims[2] < 1000:
        vol = _tiny(dims, seed, dt)
    else:
        vol = _sparse_u16(dims, seed) if dt == "u16" else _sparse_u8(dims, seed)
    st = oracle.stats(vol)
    ocfg = oracle.Config(okada_td=cfg.get("okada_td"), entropy_te=cfg.get("entropy_te"))
    kw = dict(cfg)
    if cfg.get("threshold_mode") == 1:   # a fixed threshold near the top: fewer voxels pass
        thr = int(np.percentile(vol, 99.9))
        kw["threshold_value"] = thr
        ocfg = oracle.Config(threshold_mode="fixed", threshold_value=thr)
    a = lnf.Context(**kw)
    b = _ring_context(lnf, monkeypatch, **kw)
    try:
        t = torch.from_numpy(vol).cuda()
        for r in radii:
            prm = oracle.derive_params(st, r, ocfg)
            # few enough voxels pass for the gate-first kernel to take the work
            assert np.count_nonzero(vol >= prm["T"]) * 32 <= vol.size, "volume not sparse enough"
            wants = {}
            for f in FILTERS:
                want = wants[f] = oracle.filter_volume(vol, f, r, params=prm)
                got = a.filter_volume(t, f, r).cpu().numpy()
                ring = b.filter_volume(t, f, r).cpu().numpy()
                assert np.array_equal(got, want), (f, r, int((got != want).sum()))
                assert np.array_equal(ring, want), (f, r, "ring")
            _check_multi(a, t, vol, r, prm, wants=wants)
    finally:
        a.close()
        b.close()


def test_dense_volume_leaves_the_work_to_the_ring_kernels(lnf):
    # half of the voxels pass: the gate-first kernel returns at once, the ring kernels write
    vol = phantoms.random_volume((64, 48, 40), 711, "u16")
    st = oracle.stats(vol)
    with lnf.Context() as c:
        t = torch.from_numpy(vol).cuda()
        for r in (1, 2):
            prm = oracle.derive_params(st, r)
            assert np.count_nonzero(vol >= prm["T"]) * 32 > vol.size
            for f in FILTERS:
                got = c.filter_volume(t, f, r).cpu().numpy()
                assert np.array_equal(got, oracle.filter_volume(vol, f, r, params=prm)), (f, r)
            _check_multi(c, t, vol, r, prm)


@pytest.mark.parametrize("dt", ["u16", "u8"])
def test_full_step_lists(lnf, monkeypatch, dt):
    """A volume where few voxels pass overall, but a bright block fills a
    128 x 32 x 4 region at the volume's left border (whole bitmask chunks set):
    outputs and entropies against the oracle and the ring kernels alone."""
    rng = np.random.default_rng(721)
    nx, ny, nz = 256, 128, 48
    if dt == "u16":
        vol = np.clip(np.rint(rng.normal(400, 30, (nz, ny, nx))), 0, 4095)
        vol[10:14, 32:64, 0:128] = rng.integers(2500, 3500, (4, 32, 128))
        vol[rng.random(vol.shape) < 0.002] = 4095
    else:
        vol = np.clip(np.rint(rng.normal(20, 4, (nz, ny, nx))), 0, 255)
        vol[10:14, 32:64, 0:128] = rng.integers(150, 220, (4, 32, 128))
        vol[rng.random(vol.shape) < 0.002] = 255
    vol = vol.astype(np.uint16 if dt == "u16" else np.uint8)
    st = oracle.stats(vol)
    a = lnf.Context()
    b = _ring_context(lnf, monkeypatch)
    try:
        t = torch.from_numpy(vol).cuda()
        for r in (1, 2):
            prm = oracle.derive_params(st, r)
            frac = np.count_nonzero(vol >= prm["T"]) / vol.size
            assert frac <= 1 / 32, frac
            outs, H = _check_multi(a, t, vol, r, prm)
            outs_b, H_b = b.filter_multi(t, FILTERS, r)
            for i in range(len(FILTERS)):
                assert torch.equal(outs[i], outs_b[i]), (FILTERS[i], r, "ring")
            assert np.allclose(H.cpu().numpy(), H_b.cpu().numpy(), rtol=1e-12, atol=0)
    finally:
        a.close()
        b.close()


def test_repeated_and_partial_filter_lists(lnf):
    """Filter lists with repeats (the gate-first kernel writes one output per
    filter, so a repeated list runs each filter on its own) and subsets of the
    five, all against the oracle."""
    vol = _sparse_u16((96, 40, 36), 731)
    st = oracle.stats(vol)
    prm = oracle.derive_params(st, 2)
    t = torch.from_numpy(vol).cuda()
    with lnf.Context() as c:
        for ids in ([oracle.MEAN, oracle.MEAN, oracle.SIGMA, oracle.ENTROPY, oracle.OKADA],
                    [oracle.SIGMA, oracle.OKADA], [oracle.OURS, oracle.OKADA, oracle.MEAN], [oracle.OURS],
                    [oracle.OKADA, oracle.ENTROPY, oracle.SIGMA, oracle.MEAN, oracle.OURS, oracle.SIGMA]):
            _check_multi(c, t, vol, 2, prm, ids)


@pytest.mark.parametrize("dims", [(13, 11, 7), (33, 9, 5), (40, 26, 3), (15, 9, 9)])
@pytest.mark.parametrize("dt", ["u16", "u8"])
def test_volume_tails(lnf, dt, dims):
    """Volumes whose voxel count is not a multiple of 8 or of a chunk, with
    passing voxels at the very first and last voxels, along the last row, and
    (where the volume has an interior) an interior voxel whose taps reach the
    volume's last voxel, in its last partial 16-byte vector: every filter
    against the oracle."""
    nx, ny, nz = dims
    rng = np.random.default_rng(751 + nx)
    hi = 4095 if dt == "u16" else 255
    vol = np.clip(np.rint(rng.normal(hi // 10, hi // 100, (nz, ny, nx))), 0, hi)
    vol[-1, -1, :] = hi - 3
    vol[0, 0, 0] = vol[-1, -1, -1] = hi
    if min(dims) >= 7:
        vol[-4, -4, -4] = hi - 1   # interior at r <= 2 (reach 3); its reach ends at the last voxel
    vol = vol.astype(np.uint16 if dt == "u16" else np.uint8)
    st = oracle.stats(vol)
    t = torch.from_numpy(vol).cuda()
    with lnf.Context(threshold_mode=1, threshold_value=hi // 2) as c:
        for r in (1, 2):
            prm = oracle.derive_params(st, r, oracle.Config(threshold_mode="fixed", threshold_value=hi // 2))
            assert np.count_nonzero(vol >= prm["T"]) * 32 <= vol.size
            _check_multi(c, t, vol, r, prm)


@pytest.mark.parametrize("dt,dims,seed", [("u16", (96, 40, 36), 761), ("u8", (128, 33, 29), 762),
                                          ("u16", (93, 37, 21), 763), ("u16", (9, 7, 4), 764)])
@pytest.mark.parametrize("theta", [None, int(3.2 * (1 << oracle.ENTROPY_W_BITS))])
def test_gate_local_entropy(lnf, monkeypatch, dt, dims, seed, theta):
    """The entropy filter with the cube's own grey-level probabilities (id 8)
    through the gate-first kernel (few voxels pass; each lane's cube values in
    shared memory, the levels counted by rank) against the oracle and against
    the generic kernel alone, r = 1, 2, two thresholds."""
    if dims[0] * dims[1] * dims[2] < 1000:
        vol = _tiny(dims, seed, dt)
    else:
        vol = _sparse_u16(dims, seed) if dt == "u16" else _sparse_u8(dims, seed)
    st = oracle.stats(vol)
    kw = {} if theta is None else {"entropy_local_te": theta}
    a = lnf.Context(**kw)
    b = _ring_context(lnf, monkeypatch, **kw)
    try:
        t = torch.from_numpy(vol).cuda()
        for r in (1, 2):
            prm = oracle.derive_params(st, r, oracle.Config(entropy_local_te=theta))
            assert np.count_nonzero(vol >= prm["T"]) * 32 <= vol.size, "volume not sparse enough"
            want = oracle.filter_volume(vol, oracle.ENTROPY_LOCAL, r, params=prm)
            got = a.filter_volume(t, oracle.ENTROPY_LOCAL, r).cpu().numpy()
            ring = b.filter_volume(t, oracle.ENTROPY_LOCAL, r).cpu().numpy()
            assert np.array_equal(got, want), (r, theta, int((got != want).sum()))
            assert np.array_equal(ring, want), (r, theta, "generic")
            outs, H = a.filter_multi(t, [oracle.ENTROPY_LOCAL], r)
            assert np.array_equal(outs[0].cpu().numpy(), want)
            hw = oracle.image_entropy(oracle.histogram(want))
            assert abs(float(H.cpu().numpy()[1]) - hw) <= 1e-9 * max(1.0, hw)
        a.params()
    finally:
        a.close()
        b.close()
