"""The multi-rank path of bench.py on CPU: two gloo ranks reduce their timings the way the
GPU run does (slowest rank's time, all ranks' nodes), and the seeded batches differ per
rank (weak scaling: each rank its own maps)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, nodes, launches = bench.reduce_over_ranks(100.0 + 50 * rank, 1000 * (rank + 1),
                                                      7 + rank, world, "cpu")
        out.put((rank, ms, nodes, launches))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, nodes, launches in got:
        assert ms == 150.0          # the slowest rank
        assert nodes == 3000.0      # every rank's nodes
        assert launches == 15.0


def test_one_rank_passes_through():
    import bench
    assert bench.reduce_over_ranks(5.0, 10, 3, 1, "cpu") == (5.0, 10.0, 3.0)


def test_ranks_get_distinct_batches():
    from paper_2301_00806_gb300 import instances as I
    a = I.batch_duals(64, 3, 8, seed=0 + 0)
    b = I.batch_duals(64, 3, 8, seed=0 + 1)
    assert [x.cols for x in a] != [x.cols for x in b]
