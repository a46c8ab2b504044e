"""Host-side sharding across ranks.

Instances of the batched form (one rPOD of Alg. 1 per field and parameter
sample, Sec. 4.1) share nothing, so N ranks (one GPU each) split them with no
collective on the data path: instance b goes to the rank with the
least accumulated cost, largest instances first (longest-processing-time
greedy).  The cost of an instance is its streamed work, (2q + 2) n m_b l_b.

A single large rPOD splits by rows instead (`row_blocks`): every pass over S
then ends in one sum over ranks of its small result (the Gram of the
sampled matrix, S^T Q, Q^T S), the algebra that oracle/sharded.py states and
the gloo tests check on CPU ranks.
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


def row_blocks(n: int, world: int, align: int = 64):
    """Contiguous row blocks [(row0, rows), ...] of an n-row matrix over
    `world` ranks: as even as `align`-row granularity allows (every block
    but the last starts and ends on a multiple of `align`, the row count of
    one 16-bit TMA tile), later ranks taking the extra tiles so that the
    ragged last tile sits in one of the longer blocks (block sizes differ by
    at most `align` rows); ranks beyond the tile count get empty blocks."""
    if n < 0 or world < 1 or align < 1:
        raise ValueError("need n >= 0, world >= 1, align >= 1")
    tiles = (n + align - 1) // align
    base, extra = divmod(tiles, world)
    out, t0 = [], 0
    for r in range(world):
        nt = base + (1 if r >= world - extra else 0)
        r0 = min(t0 * align, n)
        r1 = min((t0 + nt) * align, n)
        out.append((r0, r1 - r0))
        t0 += nt
    return out


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
