"""Parity of the CUDA ray caster (lnf_render, through the C ABI) with the
oracle's: image, depth and the filter value at each hit, bit for bit, for all
five filters, all six views, both dtypes; plus the image entropy of the
rendered image (the paper's Fig. 4 measure) through lnf_entropy."""
import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_03119_gb300 as L
    from paper_1807_03119_gb300 import builder
    builder.build()
    L.load()
    c = L.Context()
    yield c
    c.params()   # raises LNF_ETIMEOUT if a bounded device wait gave up
    c.close()


def _vols():
    return [("u8", phantoms.P1()),
            ("u16", phantoms.insect_phantom((45, 38, 33), 41, "u16")),
            ("u8 odd", phantoms.insect_phantom((29, 31, 27), 43, "u8", background=20, lo=40, hi=220,
                                               sigma=25.0, vmax=255))]


@pytest.mark.parametrize("f", [0, 1, 2, 3, 4])
def test_render_matches_oracle(ctx, f):
    for name, vol in _vols():
        t = torch.from_numpy(vol).cuda()
        st = oracle.stats(vol)
        for r in (1, 2):
            prm = oracle.derive_params(st, r)
            for view in range(6):
                im, d, v = ctx.render(t, f, r, view)
                torch.cuda.synchronize()
                wim, wd, wv = oracle.render(vol, f, r, view, params=prm)
                what = f"{name} filter {f} r {r} view {view}"
                assert np.array_equal(d.cpu().numpy(), wd), what + " depth"
                assert np.array_equal(v.cpu().numpy().astype(np.uint32), wv), what + " value"
                assert np.array_equal(im.cpu().numpy(), wim), what + " image"


def test_rendered_image_entropy(ctx):
    vol = phantoms.P1()
    t = torch.from_numpy(vol).cuda()
    im, _, _ = ctx.render(t, 4, 1, 4, with_depth=False, with_value=False)
    H = ctx.entropy(im.reshape(1, *im.shape).contiguous())
    wim, _, _ = oracle.render(vol, 4, 1, 4)
    want = oracle.image_entropy(np.bincount(wim.ravel(), minlength=256))
    assert abs(H - want) <= 1e-9 * max(1.0, want)
