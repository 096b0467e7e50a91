"""Multi-GPU sharding of a batch of independent configurations (weak scaling).

Configurations are independent, so N ranks (one process per GPU) split work with no exchange of
data: rank r takes configuration indices [r*B, (r+1)*B) of the workload's seeded sequence, and
the only collectives are a barrier and a max over the ranks' measured times.
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
