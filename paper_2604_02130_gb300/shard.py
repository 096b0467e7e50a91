"""Multi-GPU sharding of a batch of independent configurations (weak scaling).

Configurations are independent, so N ranks (one process per GPU) split work with no exchange of
data; the only collectives are a barrier and a max over the ranks' measured times.  A workload of
equal configurations gives rank r the indices [r*B, (r+1)*B) of its seeded sequence; a workload
of uneven sizes (different Nx and Nt) splits the first N*B indices by cost, longest first
(lpt_partition over Nx^3 Nt), so that every rank carries about the same work.
"""
from __future__ import annotations


def shard_range(rank: int, per_rank: int) -> range:
    """Configuration indices of one rank (disjoint across ranks, contiguous per rank)."""
    return range(rank * per_rank, (rank + 1) * per_rank)


def aggregate_rate(per_rank: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job configurations per second: all ranks' configurations over the slowest rank."""
    return per_rank * world * steps / (max_ms * 1e-3)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a float over all ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def lpt_partition(costs, world: int) -> list:
    """Cost-balanced split of independent configurations over `world` ranks (longest processing
    time first): configurations in order of decreasing cost, each to the rank with the smallest
    total so far (ties to the lower rank).  Returns one ascending index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]
