"""Instance sharding across GPUs (one process per GPU).

OPO instances are independent, so the multi-GPU form is data parallel with
no collective on the data path: each rank owns a contiguous block of
instance indices, runs them on its own GPU, and only scalars cross ranks
(the step time reduced by max, per-instance observables gathered on rank 0).
Works with any torch.distributed backend (gloo on CPU, NCCL on GPUs).
"""
from __future__ import annotations


def shard(total: int, world: int, rank: int) -> range:
    """Contiguous, balanced block of ``range(total)`` owned by ``rank``."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank scalar (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_to_rank0(obj, dist=None):
    """List of every rank's ``obj`` on rank 0 (None elsewhere)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return [obj]
    world = dist.get_world_size()
    out = [None] * world if dist.get_rank() == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out


__all__ = ["shard", "max_over_ranks", "gather_to_rank0"]
