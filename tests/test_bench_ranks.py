"""The multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): each
rank is an independent replica, the step time is the maximum over ranks, and
the reported throughput counts the voxels of every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = 2.0 + 3.0 * rank                     # rank 1 is the slower replica
        t = bench.max_over_ranks(ms, world, "cpu")
        v = bench.whole_job_value(1000, world, t)
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, v in res:
        assert t == 5.0                            # the slowest rank's 5 ms
        assert v == pytest.approx(2 * 1000 / 5e-3)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(1.25, 1, "cpu") == 1.25
    assert bench.whole_job_value(4096, 1, 2.0) == pytest.approx(4096 / 2e-3)
