"""Host-side logic of the multi-GPU runs (one process per GPU).

A single shot does not shard: splitting one grid across GPUs would need a
halo exchange of width r T after every pass, and the paper has no such
exchange.  Several GPUs therefore run independent replicas or independent
shots; the only collectives are a barrier and the max of the timings (and,
for a multi-shot gradient, one sum of the per-rank gradients at the end).
"""
from __future__ import annotations


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of item indices owned by `rank` (sizes differ by <= 1)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over the default process group (identity if
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(t):
    """In-place sum of a tensor over the default process group."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def job_throughput(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: units every rank processed / the slowest rank's time."""
    return units_per_rank * world / seconds_max
