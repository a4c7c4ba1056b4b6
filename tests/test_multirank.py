"""The host side of the multi-GPU path on CPU (gloo, world size 2, no GPU):
bench.py runs one replica per GPU and reports the slowest rank's time, so the
ranks' only collective is a MAX all-reduce of the timings; a rank that dies
between steps must surface as an error on the others, not a hang."""
import datetime
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, mode, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
    if mode == "max":
        q.put((rank, bench.max_over_ranks(10.0 + 3.0 * rank, world, "cpu")))
        dist.barrier()
        dist.destroy_process_group()
        return
    # mode "fail": rank 1 leaves between steps, before the next collective
    if rank == 1:
        os._exit(3)
    try:
        bench.max_over_ranks(1.0, world, "cpu")
        q.put((rank, "no error"))
    except Exception as e:   # the peer's departure must surface here
        q.put((rank, "error: " + type(e).__name__))


def _run(mode, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(60)
    for p in ps:
        if p.is_alive():
            p.kill()
            raise AssertionError(f"rank process {p.pid} still running after 60 s")
    out = {}
    while not q.empty():
        r, v = q.get()
        out[r] = v
    return out, [p.exitcode for p in ps]


@pytest.mark.timeout(120)
def test_max_over_ranks_gloo():
    out, codes = _run("max")
    assert codes == [0, 0]
    assert out == {0: 13.0, 1: 13.0}   # every rank sees the slowest rank's time


@pytest.mark.timeout(120)
def test_rank_leaving_surfaces_as_error():
    out, codes = _run("fail")
    assert codes[1] == 3
    assert 0 in out and out[0].startswith("error"), out


def test_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
