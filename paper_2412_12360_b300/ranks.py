"""Multi-GPU bookkeeping for independent problems (one process per GPU).

The solves of different designs, served requests or replicas share nothing, so N GPUs take disjoint
shares of them with no collective on the data path; only the timing is reduced (max of the ranks'
times, sum of their work) to report whole-job throughput. Works with any torch.distributed backend
(NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def shard(n_items: int, world: int, rank: int) -> List[int]:
    """Indices of the items rank `rank` of `world` solves: a contiguous, balanced block."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return list(range(lo, hi))


def reduce_time_and_work(seconds: float, units: float, device=None) -> Tuple[float, float]:
    """(max over ranks of `seconds`, sum over ranks of `units`); the local values without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds), float(units)
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def throughput(units_per_rank: Sequence[float], seconds_per_rank: Sequence[float]) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return float(sum(units_per_rank)) / float(max(seconds_per_rank))
