"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer outputs must match bit for bit; entropies within 1e-9 relative.
Small cases are compared element by element (sizes that span several tiles
with ragged tails); the full-size workloads are compared on sampled voxels
that the oracle evaluates one by one, plus properties that hold at any size.
"""
import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FILTERS = [oracle.MEAN, oracle.SIGMA, oracle.ENTROPY, oracle.OKADA, oracle.OURS]
H_TOL = 1e-9


@pytest.fixture(scope="module")
def lnf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_03119_gb300 as L
    from paper_1807_03119_gb300 import builder
    builder.build()
    L.load()
    return L


@pytest.fixture(scope="module")
def ctx(lnf):
    c = lnf.Context()
    yield c
    c.params()   # raises LNF_ETIMEOUT if any bounded device wait gave up during the module
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def assert_same(got, want, what):
    if not np.array_equal(got, want):
        idx = np.argwhere(got != want)
        z, y, x = idx[0]
        raise AssertionError(f"{what}: {len(idx)} voxels differ; first at x={x} y={y} z={z}: "
                             f"got {got[z, y, x]} want {want[z, y, x]}")


def oracle_cfg(**kw):
    mode = {0: "otsu", 1: "fixed", 2: "none"}[kw.get("threshold_mode", 0)]
    return oracle.Config(threshold_mode=mode, threshold_value=kw.get("threshold_value", 0),
                         sigma_k=kw.get("sigma_k", 2),
                         okada_td=None if kw.get("okada_td", -1) == -1 else kw["okada_td"],
                         entropy_te=None if kw.get("entropy_te", -2) == -2 else kw["entropy_te"],
                         offset=kw.get("cluster_offset", 1))


SMALL = [
    ((70, 19, 23), "u8", 101),      # 3 x-tiles, 3 y-tiles, ragged, plain loads (pitch 70 B)
    ((70, 19, 23), "u16", 102),
    ((64, 24, 40), "u16", 103),     # 16-byte pitch: TMA path
    ((96, 17, 9), "u8", 104),       # TMA path, u8
    ((40, 33, 130), "u16", 105),    # several z chunks
]


@pytest.mark.parametrize("dims,dt,seed", SMALL)
@pytest.mark.parametrize("r", [0, 1, 2, 3])
def test_small_all_filters_exact(ctx, dims, dt, seed, r):
    vol = phantoms.random_volume(dims, seed, dt, p_extreme=0.05)
    st = oracle.stats(vol)
    prm = oracle.derive_params(st, r)
    t = dev(vol)
    for f in FILTERS:
        got = host(ctx.filter_volume(t, f, r))
        want = oracle.filter_volume(vol, f, r, params=prm)
        assert_same(got, want, f"filter {f} r={r} {dims} {dt}")


@pytest.mark.parametrize("dt", ["u8", "u16"])
def test_phantom_p1_like_all_filters(ctx, dt):
    vol = phantoms.P1() if dt == "u8" else phantoms.insect_phantom((64, 48, 40), 7, "u16")
    st = oracle.stats(vol)
    t = dev(vol)
    for r in (1, 2):
        prm = oracle.derive_params(st, r)
        outs, H = ctx.filter_multi(t, FILTERS, r)
        Hh = host(H)
        assert abs(Hh[0] - oracle.image_entropy(st.hist)) <= H_TOL * max(1, Hh[0])
        for i, f in enumerate(FILTERS):
            want = oracle.filter_volume(vol, f, r, params=prm)
            assert_same(host(outs[i]), want, f"P1 filter {f} r={r}")
            hw = oracle.image_entropy(oracle.histogram(want))
            assert abs(Hh[i + 1] - hw) <= H_TOL * max(1.0, hw), (f, Hh[i + 1], hw)


def test_params_match_oracle(ctx):
    cases = [phantoms.P1(), phantoms.random_volume((33, 21, 17), 5, "u16"),
             phantoms.insect_phantom((48, 40, 36), 9, "u16"),
             np.full((5, 6, 7), 200, np.uint8), np.full((3, 4, 9), 65535, np.uint16)]
    two = np.full((8, 8, 8), 20, np.uint8)
    two[:, :, 5:] = 190
    cases.append(two)
    for vol in cases:
        t = dev(vol)
        ctx.filter_volume(t, oracle.OURS, 1)
        p = ctx.params(with_weights=True)
        st = oracle.stats(vol)
        prm = oracle.derive_params(st, 1)
        L = len(st.hist)
        assert p["n_voxels"] == st.N and p["sum"] == st.S and p["sum_sq"] == st.Q
        assert p["min_value"] == st.minv and p["max_value"] == st.maxv
        assert p["threshold"] == prm["T"], (p["threshold"], prm["T"])
        assert p["sigma_band"] == prm["delta"]
        assert p["okada_td"] == prm["td"]
        assert np.array_equal(p["weights"][:L], prm["w"]), "entropy weight tables differ"
        assert p["weight_sum"] == int(sum(int(c) * int(w) for c, w in zip(st.hist, prm["w"])))
        hin = oracle.image_entropy(st.hist)
        assert abs(p["input_entropy"] - hin) <= H_TOL * max(1.0, hin)


@pytest.mark.parametrize("kw", [
    dict(threshold_mode=2), dict(threshold_mode=1, threshold_value=150),
    dict(sigma_k=1), dict(sigma_k=3), dict(okada_td=0), dict(okada_td=40),
    dict(entropy_te=-1), dict(entropy_te=0), dict(cluster_offset=0), dict(cluster_offset=2),
])
def test_config_variants(lnf, kw):
    vol = phantoms.random_volume((45, 13, 19), 77, "u8", p_extreme=0.1)
    with lnf.Context(**kw) as c:
        t = dev(vol)
        st = oracle.stats(vol)
        for r in (1, 2):
            prm = oracle.derive_params(st, r, oracle_cfg(**kw))
            for f in FILTERS:
                assert_same(host(c.filter_volume(t, f, r)), oracle.filter_volume(vol, f, r, params=prm),
                            f"{kw} filter {f} r={r}")


def test_forced_plain_loads_match_tma(lnf, monkeypatch):
    vol = phantoms.random_volume((64, 24, 40), 31, "u16")
    t = dev(vol)
    with lnf.Context() as a:
        ref = [host(a.filter_volume(t, f, 2)) for f in FILTERS]
    monkeypatch.setenv("LNF_FORCE_PLAIN", "1")
    with lnf.Context() as b:
        got = [host(b.filter_volume(t, f, 2)) for f in FILTERS]
    for f, x, y in zip(FILTERS, ref, got):
        assert_same(y, x, f"plain vs TMA filter {f}")


def test_forced_generic_matches(lnf, monkeypatch):
    vol = phantoms.insect_phantom((80, 48, 72), 12, "u16")
    st = oracle.stats(vol)
    t = dev(vol)
    monkeypatch.setenv("LNF_FORCE_GENERIC", "1")
    with lnf.Context() as b:
        for r in (1, 2):
            prm = oracle.derive_params(st, r)
            for f in FILTERS:
                assert_same(host(b.filter_volume(t, f, r)), oracle.filter_volume(vol, f, r, params=prm),
                            f"generic filter {f} r={r}")


@pytest.mark.parametrize("dt,off", [("u8", 0), ("u8", 1), ("u8", 7), ("u8", 13), ("u16", 0), ("u16", 1),
                                    ("u16", 3)])
def test_padded_copy_of_unaligned_inputs(lnf, dt, off):
    # inputs TMA cannot address (row lengths that are not a multiple of 16 bytes,
    # bases `off` elements past a 16-byte boundary) are copied into padded rows
    # before the plane-ring kernels read them; no threshold, so those kernels do
    # the work.  Rows of 530 and 301 elements span several 512-byte segments of
    # the copy kernel; with an odd base every row starts at another offset
    # within its 16-byte block
    for dims, seed in (((530, 9, 5), 71), ((37, 23, 19), 72), ((301, 7, 6), 73)):
        vol = phantoms.random_volume(dims, seed, dt)
        n = vol.size
        padded = np.zeros(n + 16, vol.dtype)
        padded[off:off + n] = vol.ravel()
        buf = dev(padded)
        t = buf[off:off + n].view(vol.shape)
        assert (t.data_ptr() % 16 == 0) == (off == 0)
        with lnf.Context(threshold_mode=lnf.THRESH_NONE) as c:
            for f in (oracle.OURS, oracle.MEAN, oracle.SIGMA):
                got = host(c.filter_volume(t, f, 2))
                want = oracle.filter_volume(vol, f, 2, cfg=oracle_cfg(threshold_mode=2))
                assert_same(got, want, f"{dt} base +{off} dims {dims} filter {f}")


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 1, 9), (9, 1, 1), (1, 7, 1), (3, 2, 1), (17, 1, 33)])
@pytest.mark.parametrize("dt", ["u8", "u16"])
def test_degenerate_shapes(ctx, dims, dt):
    vol = phantoms.random_volume(dims, 3, dt)
    st = oracle.stats(vol)
    t = dev(vol)
    for r in (0, 1, 3):
        prm = oracle.derive_params(st, r)
        for f in FILTERS:
            assert_same(host(ctx.filter_volume(t, f, r)), oracle.filter_volume(vol, f, r, params=prm),
                        f"{dims} filter {f} r={r}")


def test_max_radius(ctx):
    vol = phantoms.random_volume((20, 18, 17), 8, "u16", vmax=3000)
    st = oracle.stats(vol)
    t = dev(vol)
    for r in (7, 8):
        prm = oracle.derive_params(st, r)
        for f in FILTERS:
            assert_same(host(ctx.filter_volume(t, f, r)), oracle.filter_volume(vol, f, r, params=prm),
                        f"max radius filter {f} r={r}")


def test_constant_volumes(ctx):
    for dt, c in (("u8", 0), ("u8", 255), ("u16", 4095), ("u16", 65535)):
        vol = np.full((11, 9, 10), c, phantoms.dtype_of(dt))
        t = dev(vol)
        for f in FILTERS:
            got = host(ctx.filter_volume(t, f, 2))
            assert (got == (0 if f == oracle.ENTROPY else c)).all(), (dt, c, f)


def test_roi_matches_crop(ctx):
    vol = phantoms.insect_phantom((77, 45, 39), 21, "u16")
    st = oracle.stats(vol)
    t = dev(vol)
    for roi in ((0, 0, 0, 77, 45, 39), (5, 3, 7, 33, 20, 11), (70, 40, 30, 7, 5, 9), (13, 0, 0, 1, 1, 1)):
        x0, y0, z0, bx, by, bz = roi
        for f in FILTERS:
            prm = oracle.derive_params(st, 2)
            got = host(ctx.filter_roi(t, f, 2, (x0, y0, z0), (bx, by, bz)))
            want = oracle.filter_volume(vol, f, 2, params=prm, roi=roi)
            assert_same(got, want, f"roi {roi} filter {f}")


def test_fast_roi_matches_oracle(ctx):
    """Regions of interest on volumes TMA can address go to the specialised
    kernels: tile grids that start left of an unaligned x origin, ROIs across
    the 128-column tile boundary, on every face of the volume, and one voxel."""
    cases = [("u16", (136, 70, 40)), ("u8", (160, 50, 36))]
    rois = [(5, 3, 7, 33, 20, 11), (120, 30, 2, 16, 40, 9), (0, 0, 0, 1, 1, 1), (127, 69, 39, 9, 1, 1),
            (1, 0, 30, 135, 9, 6)]
    for dt, dims in cases:
        if dt == "u8":
            vol = phantoms.insect_phantom(dims, 31, dt, background=20, lo=40, hi=220, sigma=25.0, vmax=255)
        else:
            vol = phantoms.insect_phantom(dims, 31, dt)
        st = oracle.stats(vol)
        t = dev(vol)
        nx, ny, nz = dims
        for x0, y0, z0, bx, by, bz in rois:
            x0, y0, z0 = min(x0, nx - 1), min(y0, ny - 1), min(z0, nz - 1)
            bx, by, bz = min(bx, nx - x0), min(by, ny - y0), min(bz, nz - z0)
            roi = (x0, y0, z0, bx, by, bz)
            for r in (1, 2, 3):
                prm = oracle.derive_params(st, r)
                for f in FILTERS:
                    got = host(ctx.filter_roi(t, f, r, (x0, y0, z0), (bx, by, bz)))
                    want = oracle.filter_volume(vol, f, r, params=prm, roi=roi)
                    assert_same(got, want, f"{dt} roi {roi} r {r} filter {f}")


def test_entropy_call(ctx):
    for vol in (phantoms.P1(), phantoms.random_volume((30, 20, 10), 4, "u16"), np.full((4, 4, 4), 9, np.uint8)):
        H = ctx.entropy(dev(vol))
        want = oracle.image_entropy(oracle.histogram(vol))
        assert abs(H - want) <= H_TOL * max(1.0, want)


def test_histogram_at_scale_with_a_dominant_level(ctx):
    """50 M voxels, 90% of them one grey level (a 12-bit one, one near 31000,
    and an 8-bit one), the rest spread over the 12-bit levels, the levels up
    to 32767 and the levels above: N, sum P, sum P^2, min, max and the image
    entropy from the device histogram against exact host sums."""
    rng = np.random.default_rng(91)
    for dt, base in (("u16", 1000), ("u16", 31000), ("u8", 77)):
        n = 512 * 512 * 192
        if dt == "u16":
            # base 1000: 12-bit data (the CTAs take the eight-copy layout of the
            # low levels); base 31000: the one-copy layout up to 32767
            vol = np.full(n, base, np.uint16)
            k = n // 10
            idx = rng.choice(n, k, replace=False)
            part = rng.integers(0, 3, k)
            vals = np.where(part == 0, rng.integers(0, 4096, k),
                            np.where(part == 1, rng.integers(4096, 32768, k), rng.integers(32768, 65536, k)))
            vol[idx] = vals.astype(np.uint16)
        else:
            vol = np.full(n, base, np.uint8)
            idx = rng.choice(n, n // 10, replace=False)
            vol[idx] = rng.integers(0, 256, n // 10).astype(np.uint8)
        vol = vol.reshape(192, 512, 512)
        t = dev(vol)
        H = ctx.entropy(t)
        ctx.filter_volume(t, oracle.OURS, 1)
        p = ctx.params()
        v64 = vol.astype(np.uint64)
        assert p["n_voxels"] == n
        assert p["sum"] == int(v64.sum()), dt
        assert p["sum_sq"] == int((v64 * v64).sum()), dt
        assert p["min_value"] == int(vol.min()) and p["max_value"] == int(vol.max()), dt
        want = oracle.image_entropy(np.bincount(vol.ravel(), minlength=65536 if dt == "u16" else 256))
        assert abs(H - want) <= H_TOL * max(1.0, want), (dt, H, want)
        del t


def test_multi_host_buffers(ctx):
    vol = phantoms.insect_phantom((48, 40, 33), 15, "u16")
    st = oracle.stats(vol)
    outs, H = ctx.filter_multi_host(vol, FILTERS, 2)
    prm = oracle.derive_params(st, 2)
    assert abs(H[0] - oracle.image_entropy(st.hist)) <= H_TOL * max(1, H[0])
    for i, f in enumerate(FILTERS):
        want = oracle.filter_volume(vol, f, 2, params=prm)
        assert_same(outs[i], want, f"host multi filter {f}")
        assert abs(H[i + 1] - oracle.image_entropy(oracle.histogram(want))) <= H_TOL * max(1, H[i + 1])


@pytest.mark.parametrize("autotune", [True, False])
def test_batched_mixed(lnf, autotune):
    # without the autotuner the first batch of a fresh context is captured
    # before any of its scratch exists: every allocation must precede the capture
    specs = phantoms.batch_volume_specs(n=6, seed=1000, lo=20, hi=60)
    vols = [phantoms.batch_volume(s) for s in specs]
    with lnf.Context(autotune=autotune) as c:
        tv = [dev(v) for v in vols]
        jobs, wants = [], []
        Hs = torch.zeros(12, dtype=torch.float64, device="cuda")
        k = 0
        for s, v, t in zip(specs, vols, tv):
            st = oracle.stats(v)
            for f in (oracle.OURS, (k % 5)):
                prm = oracle.derive_params(st, s["radius"])
                roi = None
                if k % 3 == 2:
                    nz, ny, nx = v.shape
                    roi = (1, 2, 3, nx // 2, ny // 3, nz // 2)
                out = torch.empty((roi[5], roi[4], roi[3]) if roi else v.shape, dtype=t.dtype, device="cuda")
                j = {"in": t, "out": out, "filter": f, "radius": s["radius"], "entropy": Hs[k:k + 1]}
                if roi:
                    j["roi_origin"], j["roi_dims"] = roi[:3], roi[3:]
                jobs.append(j)
                wants.append(oracle.filter_volume(v, f, s["radius"], params=prm, roi=roi))
                k += 1
        for rep in range(2):   # the second run replays the captured graph
            for j in jobs:
                j["out"].zero_()
            c.filter_batch(jobs)
            Hh = host(Hs)
            for i, (j, w) in enumerate(zip(jobs, wants)):
                assert_same(host(j["out"]), w, f"batch job {i} rep {rep}")
                hw = oracle.image_entropy(oracle.histogram(w))
                assert abs(Hh[i] - hw) <= H_TOL * max(1.0, hw), (i, Hh[i], hw)
        # the autotuner's record: one entry per class of specialised jobs, a z length
        # among the candidates, a time for every candidate
        tun = c.tuning()
        if autotune:
            assert tun["classes"], "the autotuner recorded no job class"
            for cl in tun["classes"]:
                assert cl["zlen"] in (4, 8, 16, 32) and all(v > 0 for v in cl["ms"].values()), cl
        else:
            assert not tun["classes"] and tun["generic_zchunk"] == 0


@pytest.mark.parametrize("autotune", [False, True])
def test_batched_chains_side_by_side(lnf, autotune):
    # eight whole volumes of the uneven batch workload (uint8 blobs and uint16
    # insects, 2.9-4.0 M voxels): 7, 11 and 46 pass few enough voxels for the
    # gate-first kernel to take them, the others go to the plane-ring kernels;
    # the batch runs them as job chains side by side on several streams, each
    # job with its own work counters; volume 36 also carries a mean-filter job
    # on the same chain
    pick = (4, 7, 11, 46, 19, 36, 27, 51)
    specs = [s for s in phantoms.batch_volume_specs(64) if s["index"] in pick]
    vols = [phantoms.batch_volume(s) for s in specs]
    with lnf.Context(autotune=autotune) as c:
        tv = [dev(v) for v in vols]
        jobs, wants = [], []
        Hs = torch.zeros(len(specs) + 1, dtype=torch.float64, device="cuda")
        for s, v, t in zip(specs, vols, tv):
            prm = oracle.derive_params(oracle.stats(v), s["radius"])
            fs = (oracle.OURS, oracle.MEAN) if s["index"] == 36 else (oracle.OURS,)
            for f in fs:
                k = len(jobs)
                jobs.append({"in": t, "out": torch.empty_like(t), "filter": f, "radius": s["radius"],
                             "entropy": Hs[k:k + 1]})
                wants.append(oracle.filter_volume(v, f, s["radius"], params=prm))
        for rep in range(2):   # capture, then replay
            for j in jobs:
                j["out"].fill_(7)
            c.filter_batch(jobs)
            Hh = host(Hs)
            for i, (j, w) in enumerate(zip(jobs, wants)):
                assert_same(host(j["out"]), w, f"batch job {i} rep {rep}")
                hw = oracle.image_entropy(oracle.histogram(w))
                assert abs(Hh[i] - hw) <= H_TOL * max(1.0, hw), (i, Hh[i], hw)


def test_invalid_arguments(ctx, lnf):
    t = dev(np.zeros((4, 4, 4), np.uint8))
    with pytest.raises(lnf.LnfError):
        ctx.filter_volume(t, 9, 1)              # filter ids are 0..8
    with pytest.raises(lnf.LnfError):
        ctx.filter_volume(t, 0, 9)
    with pytest.raises(lnf.LnfError):
        ctx.filter_volume(t, 0, -1)
    with pytest.raises(lnf.LnfError):
        ctx.filter_volume(t, 0, 1, out=t)       # in-place is rejected
    with pytest.raises(lnf.LnfError):
        ctx.filter_roi(t, 0, 1, (2, 2, 2), (3, 1, 1))


# ----------------------------------------------------------------------------- full sizes

def _sample_points(dims, n, seed):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    corners = [(x, y, z) for x in (0, 1, nx - 2, nx - 1) for y in (0, ny - 1) for z in (0, 2, nz - 1)]
    pts = np.stack([rng.integers(0, nx, n), rng.integers(0, ny, n), rng.integers(0, nz, n)], axis=1)
    return np.concatenate([np.array(corners), pts]).astype(np.int64)


def _check_sampled(vol, outs, filters, r, prm, seed):
    nz, ny, nx = vol.shape
    pts = _sample_points((nx, ny, nz), 3000, seed)
    for f, o in zip(filters, outs):
        want = oracle.filter_points(vol, f, r, pts, prm)
        got = o[pts[:, 2], pts[:, 1], pts[:, 0]]
        bad = np.nonzero(got != want)[0]
        assert bad.size == 0, (f, pts[bad[:5]], got[bad[:5]], want[bad[:5]])


def _check_slabs(vol, outs, filters, r, prm, planes):
    """Whole z-planes: every voxel below the noise threshold T must be 0, and
    every voxel with P0 >= T is checked against the oracle element by element
    (the planes include the volume's first and last ones, where the clamped
    taps run)."""
    T = prm["T"]
    checked = 0
    for z in planes:
        sl = vol[z]
        ys, xs = np.nonzero(sl >= T)
        pts = np.stack([xs, ys, np.full_like(xs, z)], axis=1).astype(np.int64)
        for f, o in zip(filters, outs):
            assert not o[z][sl < T].any(), (f, z, "nonzero below the gate")
            if len(pts):
                want = oracle.filter_points(vol, f, r, pts, prm)
                got = o[z][ys, xs]
                bad = np.nonzero(got != want)[0]
                assert bad.size == 0, (f, z, pts[bad[:5]], got[bad[:5]], want[bad[:5]])
        checked += len(pts)
    assert checked > 0
    return checked


def _check_hist_property(out, Hgot):
    # the fused output histogram must be the histogram of the output
    h = np.bincount(out.reshape(-1).astype(np.int64))
    hw = oracle.image_entropy(h)
    assert abs(Hgot - hw) <= H_TOL * max(1.0, hw)


def test_full_512_u16_all_filters_r2(ctx):
    """The 512^3 uint16 insect phantom, all five filters at radius 2, entropy of
    input and outputs, in the launch configuration the benchmark times: 3000
    random voxels, and every voxel of nine whole z-planes."""
    vol = phantoms.P2()
    st = oracle.stats(vol)
    prm = oracle.derive_params(st, 2)
    t = dev(vol)
    outs, H = ctx.filter_multi(t, FILTERS, 2)
    Hh = host(H)
    p = ctx.params()
    assert p["threshold"] == prm["T"] and p["sigma_band"] == prm["delta"] and p["okada_td"] == prm["td"]
    assert abs(Hh[0] - oracle.image_entropy(st.hist)) <= H_TOL * Hh[0]
    outs_h = [host(o) for o in outs]
    _check_sampled(vol, outs_h, FILTERS, 2, prm, 5)
    # whole planes within the reach (3) of both z faces and one in the middle
    _check_slabs(vol, outs_h, FILTERS, 2, prm, (0, 1, 2, 3, 256, 508, 509, 510, 511))
    for o, h in zip(outs_h, Hh[1:]):
        _check_hist_property(o, h)


def test_full_1024_u8_ours_radius_sweep(ctx):
    vol = phantoms.P3()
    st = oracle.stats(vol)
    t = dev(vol)
    for r in (1, 2, 3, 4):
        prm = oracle.derive_params(st, r)
        outs, H = ctx.filter_multi(t, [oracle.OURS], r)
        o = host(outs[0])
        _check_sampled(vol, [o], [oracle.OURS], r, prm, 10 + r)
        _check_slabs(vol, [o], [oracle.OURS], r, prm, (0, r + 1, 511, 1022 - r, 1023))
        _check_hist_property(o, float(host(H)[1]))
        del outs, o
        torch.cuda.empty_cache()


def test_largest_accepted_volume(lnf):
    """2048 x 2048 x 1023 uint8 = 4,290,772,992 voxels, just under the API's limit
    of 2^32 - 1 (32-bit voxel indices in the gate-first kernel, 64-bit offsets
    elsewhere): the statistics against the host, the paper's filter through the
    gate-first kernel (0.6% of the voxels pass) and, with no noise threshold,
    through the plane-ring kernel, each on sampled voxels and whole first and last
    planes against the oracle; a volume of exactly 2^32 voxels is refused."""
    nx, ny, nz = 2048, 2048, 1023
    rng = np.random.default_rng(99)
    vol = rng.integers(0, 40, size=(nz, ny, nx), dtype=np.uint8)
    vol[100:140, 500:1000, 500:1500] = 200          # 0.47% of the voxels
    vol[nz - 40:, ny - 200:, nx - 600:] = 210        # up to the last plane, row and column
    vol[:2, :300, :64] = 220                         # in the first planes
    st = oracle.stats(vol)
    t = dev(vol)
    for mode in (0, 2):   # Otsu (gate-first kernel), none (plane-ring kernel)
        cfg = oracle.Config(threshold_mode="otsu" if mode == 0 else "none")
        prm = oracle.derive_params(st, 1, cfg)
        if mode == 0:
            assert np.count_nonzero(vol >= prm["T"]) * 32 <= vol.size
        with lnf.Context(threshold_mode=mode) as c:
            out = c.filter_volume(t, oracle.OURS, 1)
            p = c.params()
            assert p["n_voxels"] == vol.size and p["sum"] == st.S and p["sum_sq"] == st.Q
            assert p["threshold"] == prm["T"]
            o = host(out)
            del out
        _check_sampled(vol, [o], [oracle.OURS], 1, prm, 41 + mode)
        _check_slabs(vol, [o], [oracle.OURS], 1, prm, (0, 1, nz - 2, nz - 1))
        del o
    del t
    torch.cuda.empty_cache()
    big = torch.empty((1024, 2048, 2048), dtype=torch.uint8, device="cuda")   # 2^32 voxels
    with lnf.Context() as c:
        with pytest.raises(lnf.LnfError) as e:
            c.filter_volume(big, oracle.OURS, 1)
        assert e.value.status == 1
    del big
    torch.cuda.empty_cache()


# ----------------------------------------------------------------------------- specialised kernels

FAST_CASES = [
    ((272, 72, 40), "u16", "narrow"),   # 3 x-tiles and 3 y-tiles (ragged), 3 z chunks
    ((272, 72, 40), "u16", "wide"),     # full 16-bit range: unpacked pairs
    ((288, 40, 33), "u8", "narrow"),
    ((128, 32, 17), "u16", "narrow"),   # exactly one tile
    ((16, 8, 5), "u16", "wide"),        # smaller than a tile in every direction
    ((32, 130, 7), "u8", "narrow"),
]


@pytest.mark.parametrize("dims,dt,kind", FAST_CASES)
def test_fast_ours_matches_oracle(ctx, dims, dt, kind):
    if kind == "narrow":
        vol = (phantoms.insect_phantom(dims, 41, dt) if dt == "u16"
               else phantoms.ellipsoid_phantom(dims, 41, dt))
    else:
        vol = phantoms.random_volume(dims, 42, dt, p_extreme=0.2)
    st = oracle.stats(vol)
    t = dev(vol)
    for r in (1, 2, 3, 4):
        prm = oracle.derive_params(st, r)
        outs, H = ctx.filter_multi(t, [oracle.OURS], r)
        want = oracle.filter_volume(vol, oracle.OURS, r, params=prm)
        assert_same(host(outs[0]), want, f"fast ours r={r} {dims} {dt} {kind}")
        hw = oracle.image_entropy(oracle.histogram(want))
        assert abs(float(host(H)[1]) - hw) <= H_TOL * max(1.0, hw)


@pytest.mark.parametrize("dt", ["u8", "u16"])
def test_tap_kernels_sparse_and_dense_warps(ctx, dt):
    # sigma and Okada evaluate only the voxels with P0 >= T when every lane of a
    # warp holds few of them, and every voxel otherwise: one volume whose upper
    # half is a phantom (mostly below T: sparse warps, with isolated salt) and
    # whose lower half is uniform noise (dense warps) exercises both forms and
    # the warps at their boundary
    dims = (136, 70, 23)
    if dt == "u16":
        vol = phantoms.insect_phantom(dims, 91, dt)
    else:
        vol = phantoms.ellipsoid_phantom(dims, 91, dt)
    noise = phantoms.random_volume(dims, 92, dt, p_extreme=0.1)
    vol[:, 35:, :] = noise[:, 35:, :]
    vol[:, 20:23, 40:44] = np.iinfo(vol.dtype).max   # a dense clump inside the sparse half
    st = oracle.stats(vol)
    t = dev(vol)
    for r in (1, 2, 3, 4):
        prm = oracle.derive_params(st, r)
        for f in (oracle.SIGMA, oracle.OKADA):
            got = host(ctx.filter_volume(t, f, r))
            assert_same(got, oracle.filter_volume(vol, f, r, params=prm), f"tap filter {f} r={r} {dt}")
