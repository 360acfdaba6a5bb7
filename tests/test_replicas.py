"""Replica (query-parallel) host logic with two gloo ranks on the CPU."""

import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2506_16488_gb300.replicas import max_over_ranks, rank_seed, shard, sum_over_ranks


def test_shards_cover_every_query_once():
    pairs = np.arange(2 * 101).reshape(-1, 2)
    for world in (1, 2, 3, 8):
        parts = [shard(pairs, r, world) for r in range(world)]
        assert np.array_equal(np.concatenate(parts), pairs)
        assert max(p.shape[0] for p in parts) - min(p.shape[0] for p in parts) <= 1
    assert rank_seed(2002, 0) == 2002 and rank_seed(2002, 1) != rank_seed(2002, 0)


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank "times" its own shard; the step time is the slowest rank's
    t = max_over_ranks(10.0 + rank)
    q = sum_over_ranks(shard(np.arange(2 * 1000).reshape(-1, 2), rank, world).shape[0])
    out.put((rank, t, q))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_queries():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]
    assert [r[2] for r in res] == [1000.0, 1000.0]
