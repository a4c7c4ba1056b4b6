"""float32 volumes on the GPU (65536 levels spanning the range, float32
rounding at every step): bit-exact with the oracle for every filter, isotropic
and anisotropic, on sizes with ragged tails; non-finite volumes are refused."""
import numpy as np
import pytest

import oracle

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


def _ct_like(shape, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, 40.0, shape).astype(np.float32) - np.float32(1000.0)
    v[shape[0] // 4:, shape[1] // 4:, :] += np.float32(1040.0)
    v[shape[0] // 2:, :, shape[2] // 3:] += np.float32(2200.5)
    salt = rng.random(shape) < 0.01
    v[salt] = np.float32(3071.0)
    return v.astype(np.float32)


@pytest.mark.parametrize("shape,seed", [((19, 37, 70), 601), ((24, 40, 128), 602), ((17, 33, 45), 603)])
def test_f32_matches_oracle(lnf, shape, seed):
    v = _ct_like(shape, seed)
    d = torch.from_numpy(v).cuda()
    with lnf.Context() as c:
        for f in range(8):
            for r, off in ((2, None), ((2, 1, 1), (1, 1, 2))):
                got = c.filter_volume_f32(d, f, r, off).cpu().numpy()
                want = oracle.filter_volume_f32(v, f, r, offset=off)
                assert np.array_equal(got, want), (f, r, off, int((got != want).sum()))


def test_f32_constant_and_refusals(lnf):
    with lnf.Context() as c:
        v = torch.full((9, 10, 11), 5.5, dtype=torch.float32, device="cuda")
        assert (c.filter_volume_f32(v, lnf.OURS, 1) == 5.5).all()
        for bad in (float("nan"), float("inf")):
            w = v.clone()
            w[3, 4, 5] = bad
            with pytest.raises(lnf.LnfError) as e:
                c.filter_volume_f32(w, lnf.MEAN, 1)
            assert e.value.status == 1
        w = v.clone()
        w[0, 0, 0], w[1, 1, 1] = -3e38, 3e38   # the span overflows float32
        with pytest.raises(lnf.LnfError) as e:
            c.filter_volume_f32(w, lnf.MEAN, 1)
        assert e.value.status == 1
