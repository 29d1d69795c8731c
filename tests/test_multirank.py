"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

Each rank runs an independent replica (no exchange step on the data path);
the only collective is the max-over-ranks of the timed region, and the
reported rate is the units all ranks processed over the slowest rank's time.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_setup()
        seconds = [2.0, 3.0][r]                       # rank 1 is the slow one
        slowest = bench.max_over_ranks(seconds, w)
        out[r] = (w, r, local, slowest, bench.aggregate_rate(1000.0, w, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_with_the_slowest_time():
    port = _free_port()
    manager = mp.get_context("spawn").Manager()  # no fork of a process that may run threads
    out = manager.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        w, rank, local, slowest, rate = out[r]
        assert (w, rank, local) == (2, r, r)
        assert slowest == 3.0
        assert rate == pytest.approx(2 * 1000.0 / 3.0)


def test_single_rank_needs_no_collective():
    assert bench.max_over_ranks(1.5, 1) == 1.5
    assert bench.aggregate_rate(10.0, 1, 2.0) == 5.0
