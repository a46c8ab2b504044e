"""Host-side sharding of independent rPOD instances across ranks.

Instances of the batched form share nothing, so N ranks (one GPU each) split
them with no collective on the data path: instance b goes to the rank with the
least accumulated cost, largest instances first (longest-processing-time
greedy).  The cost of an instance is its streamed work, (2q + 2) n m_b l_b.
"""
from __future__ import annotations


def instance_cost(n: int, m: int, k: int, p: int, q: int) -> float:
    return float(2 * q + 2) * n * m * (k + p)


def shard(costs, world: int):
    """List of instance-index lists, one per rank; every index appears once."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda j: (load[j], j))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, group=None) -> float:
    """The largest of the ranks' values (the timing rule: the slowest rank
    sets the step time).  Plain float when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
