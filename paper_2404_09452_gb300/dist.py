"""Multi-GPU helpers.  Molecules (and requests) are independent units, so
ranks split them with no data-path collective; the only collectives are the
timing barrier and the max over ranks of the elapsed time."""

from __future__ import annotations


def shard_round_robin(n: int, rank: int, world: int):
    """Indices of the n units that `rank` of `world` processes."""
    return list(range(rank, n, world))


def shard_balanced(costs, world: int):
    """Longest-processing-time assignment: per rank, the unit indices, so that
    the per-rank summed cost is balanced (costs e.g. atoms^3)."""
    loads = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: -costs[k]):
        r = min(range(world), key=lambda q: loads[q])
        out[r].append(i)
        loads[r] += costs[i]
    return [sorted(x) for x in out]


def max_over_ranks(value: float, device=None) -> float:
    """Max of `value` over the ranks of the default process group (value
    itself without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
