"""Instance sharding across ranks (one process per GPU).

The (n, d) instances of a sweep are independent BA problems, so N ranks split
the instance list and exchange nothing on the data path; only the timing
(max over ranks) and the per-instance results (gathered to rank 0) cross
process boundaries, through torch.distributed (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import List, Sequence


def shard(items: Sequence, rank: int, world: int) -> List:
    """Round-robin share of `items` owned by `rank` (every item exactly once)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    return list(items[rank::world])


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar (e.g. the timed region in ms)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_to_rank0(obj):
    """All ranks' objects as a list on rank 0 (None elsewhere)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out
