"""The multi-GPU path of the benchmark is replicas only (each rank solves its own copy; the
path has no exchange step): step time = maximum over ranks, work = sum over ranks.  This
checks that reduction with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.over_ranks(10.0 + 5.0 * rank, "max")          # rank 1 is the slower replica
        work = bench.over_ranks(1000.0 * (rank + 1), "sum")
        ws, r, _ = bench.dist_env()
        out[rank] = (ms, work, ws, r)
    finally:
        dist.destroy_process_group()


def test_replicas_reduce_time_by_max_and_work_by_sum():
    world = 2
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        ms, work, ws, r = out[rank]
        assert ms == 15.0 and work == 3000.0 and ws == world and r == rank


def test_single_process_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.over_ranks(7.5, "max") == 7.5 and bench.over_ranks(3.0, "sum") == 3.0
