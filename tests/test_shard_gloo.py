"""Multi-rank host logic on CPU: sharding of independent instances and the
max-over-ranks timing reduction, with two gloo ranks."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2504_15350_gb300.shard import instance_cost, max_over_ranks, shard
from synth import batched_recipes


def test_shard_covers_all_once_and_balances():
    recs, ks = batched_recipes(count=64, nx=128, ny=256, J=20, seed=0)
    costs = [instance_cost(r.n, r.m, k, 10, 1) for r, k in zip(recs, ks)]
    for world in (1, 2, 3, 4, 8):
        parts = shard(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy bound: no rank exceeds the mean by more than the largest instance
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-6


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
        recs, ks = batched_recipes(count=16, nx=32, ny=32, J=10, seed=1)
        costs = [instance_cost(r.n, r.m, k, 10, 1) for r, k in zip(recs, ks)]
        mine = shard(costs, world)[rank]
        t = max_over_ranks(1.0 + rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out[rank] = (t, sorted(i for g in gathered for i in g))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, union = res[rank]
        assert t == 2.0                     # the slowest rank's value
        assert union == list(range(16))     # disjoint shards cover every instance
