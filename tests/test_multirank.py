"""Multi-process host logic of bench.py on CPU ranks (gloo, world size 2).

The bench runs one replica of the workload per rank (the workload is a single
problem; there is no data-path collective).  The whole-job time is the max
over ranks and the work is the sum, so value = total passes / slowest rank.
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times = [10.0 + 5.0 * rank, 1.0 + rank]          # rank 1 is slower
        counts = [61.0, 61.0 + rank, 7.0]
        t, c = bench.aggregate_over_ranks(times, counts, dist, "cpu")
        out[rank] = (t, c)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        res = dict(out)
    for r in range(world):
        t, c = res[r]
        assert t == [15.0, 2.0]                            # max over ranks
        assert c == [122.0, 123.0, 14.0]                   # sums over ranks


def test_aggregate_single_process_is_identity():
    t, c = bench.aggregate_over_ranks([3.0, 4.0], [5, 6], None, "cpu")
    assert t == [3.0, 4.0] and c == [5.0, 6.0]
