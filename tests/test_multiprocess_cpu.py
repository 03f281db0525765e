"""The N > 1 launch paths of bench.py, on CPU with gloo (world size 2).

The code path runs independent replicas, one per GPU (no collective in the
data path; each rank learns its own frame).  What crosses ranks is the
timing: the whole-job time is the slowest rank's (max over ranks), and only
rank 0 prints.  These tests run that aggregation over two gloo ranks, and
check that a non-zero rank of the reference arm returns at once without work.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                  # each rank's own time
        out[rank] = bench.max_over_ranks(ms, world)
        w, r, local = bench._dist()
        assert (w, r, local) == (world, rank, rank)
        if rank == 1:
            class A:  # the reference arm's arguments; rank 1 must not run the oracle
                steps, warmup = 1, 0
            assert bench.run_reference(A()) is None
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_reference_rank_exit():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1] == 15.0     # every rank sees the slowest rank's time


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
