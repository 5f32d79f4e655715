"""The N > 1 bookkeeping of bench.py on CPU ranks (gloo, world size 2).

With several GPUs the stencil and R-MAT workloads run replicas and the
batched workload shards its independent instances over the ranks; neither
has a data-path collective.  What the ranks share is the timing: the job's
rate is all ranks' units over the slowest rank's time.  These tests run that
reduction and the sharding with two gloo processes.
"""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, local_ms, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = (bench.slowest_rank_ms(dist, local_ms[rank], "cpu"), bench.shard_units(256, rank, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_sharding_with_two_gloo_ranks():
    world = 2
    local_ms = [12.5, 40.25]
    # spawn, not fork: the test process may already run threads (the
    # oracle's OpenMP pool), which a forked child must not inherit
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), local_ms, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 40.25
    shards = [res[r][1] for r in range(world)]
    assert sorted(shards[0] + shards[1]) == list(range(256))
    assert not set(shards[0]) & set(shards[1])
    assert abs(len(shards[0]) - len(shards[1])) <= 1


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.slowest_rank_ms(None, 3.5, "cpu") == 3.5
    assert bench.shard_units(5, 0, 1) == [0, 1, 2, 3, 4]
