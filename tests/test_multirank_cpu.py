"""The N>1 path of bench.py on CPU ranks (gloo, world size 2): ensemble
boxes are sharded with no data-path communication (every box owned by
exactly one rank), the job time is the slowest rank's, and the job rate
counts the units of all ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = bench.shard(24, rank, world)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = bench.reduce_max(1.0 + rank, dist, "cpu")     # rank 1 is slower
        rate = bench.job_throughput(100.0, world, t)
        out[rank] = (gathered, t, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        gathered, t, rate = out[rank]
        owned = sorted(i for part in gathered for i in part)
        assert owned == list(range(24))                       # each box exactly once
        assert set(gathered[0]).isdisjoint(gathered[1])
        assert t == 2.0                                       # slowest rank
        assert rate == pytest.approx(100.0 * 2 / 2.0)
