"""Instance sharding across ranks (one process per GPU).

The (n, d) instances of a sweep are independent BA problems, so N ranks split
the instance list and exchange nothing on the data path; only the timing
(max over ranks) and the per-instance results (gathered to rank 0) cross
process boundaries, through torch.distributed (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import Dict, List, Sequence


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


def shard_grid(grid: Dict[int, Sequence[float]], rank: int, world: int) -> Dict[int, List[float]]:
    """Share of a workload grid {n: [d, ...]} owned by `rank`: every (n, d)
    instance goes to exactly one rank.  Instances are placed largest first
    (one iteration costs about 2^n), each on the rank with the least work so
    far (ties to the lowest rank), so shares of mixed sizes balance.  Returns
    {n: [d, ...]} in the grid's order, without the sizes the rank does not
    own."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    items = [(n, i, d) for n, ds in grid.items() for i, d in enumerate(ds)]
    order = sorted(items, key=lambda t: (-t[0], t[1]))
    load = [0] * world
    owner = {}
    for n, i, d in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[(n, i)] = r
        load[r] += 1 << n
    out: Dict[int, List[float]] = {}
    for n, ds in grid.items():
        mine = [d for i, d in enumerate(ds) if owner[(n, i)] == rank]
        if mine:
            out[n] = mine
    return out


def init_from_env(backend: str = "nccl"):
    """(rank, world) from torchrun's environment; initialises the process
    group when world > 1 (NCCL for GPU ranks, gloo for host-only runs)."""
    import os
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return rank, world
