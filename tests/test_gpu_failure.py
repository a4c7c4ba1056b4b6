"""Failure detection on the GPU without a GPU fault: a bounded device wait on
a barrier that nothing completes must give up after its limit, report
LNF_ETIMEOUT through the host, and leave the context usable."""
import numpy as np
import pytest

import oracle
import phantoms

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ETIMEOUT, EINVAL = 6, 1


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
