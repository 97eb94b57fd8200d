"""The multi-GPU mode of bench.py is N independent replicas (the solve does not shard): every
rank runs the whole workload, the ranks meet at a barrier, the time is the slowest rank's and
the value counts the units of all ranks.  Checked on the CPU with two gloo ranks on
127.0.0.1: max_over_ranks gives every rank the largest time, replica_throughput the
whole-job rate, and one rank needs no process group."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        assert (r, w, lr) == (rank, world, rank)
        dist.barrier()
        my_ms = 10.0 + 5.0 * rank                     # rank 1 is the slower one
        slowest = bench.max_over_ranks(my_ms, world)
        out.put((rank, slowest, bench.replica_throughput(8 * 20, world, slowest / 1e3)))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, value in res:
        assert slowest == 15.0
        assert value == pytest.approx(2 * 160 / 0.015)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_throughput(160, 1, 0.5) == 320.0
