"""Replica runs of bench.py (one solve stream per rank, no data-path
collective): the whole-job rate is every rank's solves over the slowest
rank's time.  Checked with two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, lists, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.whole_job_rate(lists[rank], 1000, world, True, "cpu")))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    world = 2
    lists = [[2.0, 2.0, 2.0], [3.0, 1.0, 4.0]]      # 6 ms and 8 ms: rank 1 is slower
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, lists, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = (world * 3 * 1000 / (8.0 / 1e3), 8.0 / 3)
    for r in range(world):
        assert out[r][0] == pytest.approx(expect[0]) and out[r][1] == pytest.approx(expect[1])
    # one rank alone: its own time
    import bench
    assert bench.whole_job_rate([2.0, 2.0], 500, 1, False, "cpu") == pytest.approx((2 * 500 / 4e-3, 2.0))
