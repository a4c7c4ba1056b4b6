"""Failure detection on the GPU without a GPU fault.

A bounded device wait on a barrier that nothing completes must give up after
its limit, report LNF_ETIMEOUT through the host, and leave the context usable.
Host-side fault injection (LNF_FAULT, read when a context is created) makes an
allocation or a launch report failure where the real call would: each site
must return its documented status, give back what it held, and leave the
context able to serve the next call bit-exactly."""
import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ETIMEOUT, EINVAL, ENOMEM, ECUDA = 6, 1, 2, 5


@pytest.fixture(scope="module")
def lnf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1807_03119_gb300 as L
    from paper_1807_03119_gb300 import builder
    builder.build()
    L.load()
    return L


def test_bounded_wait_gives_up_and_the_context_survives(lnf):
    with lnf.Context() as c:
        for limit in (20.0, 80.0):
            rc, ms = c.selftest_wait(limit)
            assert rc == ETIMEOUT
            assert limit <= ms < limit + 1000.0, ms
        # the same context still filters correctly afterwards
        vol = phantoms.P1()
        got = c.filter_volume(torch.from_numpy(vol).cuda(), oracle.OURS, 1).cpu().numpy()
        assert np.array_equal(got, oracle.filter_volume(vol, oracle.OURS, 1))
        c.params()   # the filters' own status word is untouched
        rc, _ = c.selftest_wait(0.0)
        assert rc == EINVAL


def _ctx(lnf, monkeypatch, spec, **kw):
    monkeypatch.setenv("LNF_FAULT", spec)
    try:
        return lnf.Context(**kw)
    finally:
        monkeypatch.delenv("LNF_FAULT")


def test_injected_scratch_failure_fails_create(lnf, monkeypatch):
    with pytest.raises(lnf.LnfError) as e:
        _ctx(lnf, monkeypatch, "scratch@1")
    assert e.value.status == ENOMEM
    with lnf.Context() as c:   # nothing was left behind
        vol = phantoms.P1()
        got = c.filter_volume(torch.from_numpy(vol).cuda(), oracle.MEAN, 1).cpu().numpy()
        assert np.array_equal(got, oracle.filter_volume(vol, oracle.MEAN, 1))


def test_injected_resident_failure_restores_the_budget(lnf, monkeypatch):
    vol = phantoms.insect_phantom((40, 36, 30), 3101, "u16")
    with _ctx(lnf, monkeypatch, "resident@1") as c:
        with pytest.raises(lnf.LnfError) as e:
            c.register_volume(vol)
        assert e.value.status == ENOMEM
        assert c.serving_stats()["budget_used"] == 0
        vid = c.register_volume(vol)   # the second attempt is not injected
        out = np.zeros_like(vol)
        tk = c.submit(vid, oracle.OURS, 2, out_host=out)
        assert c.wait(tk).status == 0
        c.release(tk)
        assert np.array_equal(out, oracle.filter_volume(vol, oracle.OURS, 2))


@pytest.mark.parametrize("site,status", [("output", ENOMEM), ("launch", ECUDA)])
def test_injected_request_failure_fails_only_that_request(lnf, monkeypatch, site, status):
    vol = phantoms.insect_phantom((48, 40, 36), 3102, "u16")
    # one request in flight at a time: each request is its own wave
    with _ctx(lnf, monkeypatch, site + "@2", max_inflight=1) as c:
        vid = c.register_volume(vol)
        resident = c.serving_stats()["budget_used"]
        outs = [np.zeros_like(vol) for _ in range(3)]
        tks = [c.submit(vid, oracle.SIGMA, 2, out_host=o, want_entropy=True) for o in outs]
        res = [c.wait(tk) for tk in tks]
        assert [r.status for r in res] == [0, status, 0]
        want = oracle.filter_volume(vol, oracle.SIGMA, 2)
        assert np.array_equal(outs[0], want) and np.array_equal(outs[2], want)
        H = oracle.image_entropy(oracle.histogram(want))
        for r in (res[0], res[2]):
            assert abs(r.entropy - H) <= 1e-9 * max(1.0, H)
        with pytest.raises(lnf.LnfError):
            c.result_copy(tks[1], np.zeros_like(vol))   # a failed request has no result
        for tk in tks:
            c.release(tk)
        st = c.serving_stats()
        assert st["budget_used"] == resident and st["inflight"] == 0 and st["queued"] == 0
        c.unregister_volume(vid)


def test_injected_launch_failure_on_a_plain_call(lnf, monkeypatch):
    vol = phantoms.insect_phantom((40, 36, 30), 3103, "u16")
    d = torch.from_numpy(vol).cuda()
    with _ctx(lnf, monkeypatch, "launch@1") as c:
        with pytest.raises(lnf.LnfError) as e:
            c.filter_volume(d, oracle.OKADA, 1)
        assert e.value.status == ECUDA
        got = c.filter_volume(d, oracle.OKADA, 1).cpu().numpy()
        assert np.array_equal(got, oracle.filter_volume(vol, oracle.OKADA, 1))


def test_injected_stage_failure_falls_back_to_the_generic_kernel(lnf, monkeypatch):
    # rows of 37 u16 voxels (74 bytes) are not TMA-addressable: the plain and
    # batched calls copy such a volume to padded rows; without room for that
    # copy the generic kernel reads the input itself, with the same result
    vol = phantoms.insect_phantom((37, 33, 29), 3104, "u16")
    d = torch.from_numpy(vol).cuda()
    for f in (oracle.OURS, oracle.SIGMA, oracle.MEAN):
        want = oracle.filter_volume(vol, f, 2)
        with _ctx(lnf, monkeypatch, "stage") as c:
            assert np.array_equal(c.filter_volume(d, f, 2).cpu().numpy(), want)
            out = torch.empty_like(d)
            c.filter_batch([{"in": d, "out": out, "filter": f, "radius": 2}])
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), want)
