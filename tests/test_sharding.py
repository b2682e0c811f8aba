"""Multi-rank host logic on CPU with the gloo backend (world size 2): shot sharding covers
every shot exactly once with balanced cost, and the timing reductions agree on all ranks."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1808_10481_gb300.sharding import max_over_ranks, shard_by_cost, sum_over_ranks


def test_shard_by_cost_partitions_and_balances():
    costs = [n * n for n in (128, 1024, 300, 777, 512, 640, 900, 200, 1000, 129)]
    for world in (1, 2, 3, 4):
        parts = shard_by_cost(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)      # LPT bound
    assert shard_by_cost(costs, 2) == shard_by_cost(list(costs), 2)   # deterministic


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, costs, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard_by_cost(costs, world)[rank]
        work = float(sum(costs[i] for i in mine))
        total = sum_over_ranks(work, dist)
        slowest = max_over_ranks(10.0 + rank, dist)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, mine, total, slowest, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_shards_and_reductions():
    costs = [n * n for n in (256, 1024, 640, 130, 990, 512, 333)]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    shards = [r[1] for r in results]
    assert sorted(i for s in shards for i in s) == list(range(len(costs)))
    for rank, mine, total, slowest, gathered in results:
        assert total == float(sum(costs))
        assert slowest == 11.0
        assert gathered == shards
