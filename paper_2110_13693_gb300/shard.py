"""Weak-scaling split of candidate plans over ranks (one process per GPU).

Plans are independent (each is scored on its own, Sec. 5, Eq. (2)), so ranks
share nothing on the data path: rank r scores its own plan batches, whose
generator plan indices start at (r * batches_per_rank + b) * plans_per_batch.
Only the timing is combined: the job time is the slowest rank's, the work is
the sum over ranks.
"""
from __future__ import annotations


def plan_base(rank: int, batch: int, batches_per_rank: int, plans_per_batch: int) -> int:
    """First generator plan index of batch `batch` of rank `rank`."""
    if rank < 0 or batch < 0 or batch >= batches_per_rank:
        raise ValueError("rank/batch out of range")
    return (rank * batches_per_rank + batch) * plans_per_batch


def plan_ranges(world: int, batches_per_rank: int, plans_per_batch: int):
    """[(rank, batch, first, last+1)] over all ranks: disjoint, covering."""
    return [(r, b, plan_base(r, b, batches_per_rank, plans_per_batch),
             plan_base(r, b, batches_per_rank, plans_per_batch) + plans_per_batch)
            for r in range(world) for b in range(batches_per_rank)]


def combine(elapsed_ms: float, work: float, device=None):
    """(max elapsed over ranks, total work over ranks) through torch.distributed
    when a process group is initialised, else the local values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_ms), float(work)
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())
