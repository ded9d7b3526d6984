"""Weak-scaling split of candidate plans over ranks (one process per GPU).

Plans are independent (each is scored on its own, Sec. 5, Eq. (2)), so ranks
share nothing on the data path: rank r scores its own plan batches, whose
generator plan indices start at (r * batches_per_rank + b) * plans_per_batch.
The timing is combined (the job time is the slowest rank's, the work the sum
over ranks); the results are exchanged once, after scoring: an all-gather of
the int64 plan costs (``gather_plan_costs``) or of each rank's cheapest
(cost, plan) pair (``best_plan``).
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


def _group_size():
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 1
    return dist.get_world_size()


def gather_plan_costs(local):
    """All-gather of per-plan int64 costs: every rank passes the costs of its
    own contiguous plan range (a [n_r] or [n_r, k] int64 tensor, n_r may
    differ between ranks, ranks in plan order) and receives the costs of all
    plans in plan order.  This is the one exchange the plan split needs
    (Sec. 5, Eq. (2): each plan is scored on its own, so only the results
    move).  Without a process group it returns `local`."""
    import torch
    import torch.distributed as dist
    if _group_size() == 1:
        return local
    if local.dtype != torch.int64:
        raise ValueError("plan costs are int64")
    world = dist.get_world_size()
    n = torch.tensor([local.shape[0]], dtype=torch.int64, device=local.device)
    counts = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(counts, n)
    counts = [int(c.item()) for c in counts]
    width = max(counts)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=torch.int64, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


def best_plan(local_costs, first_plan: int):
    """(cost, plan index) of the cheapest plan over all ranks, ties to the
    lowest plan index: each rank takes its own minimum over the int64 costs
    of plans first_plan .. first_plan + n_r - 1, then one all-gather of the
    (cost, plan) pairs picks the global one.  A rank with no plans passes an
    empty tensor."""
    import torch
    import torch.distributed as dist
    big = torch.iinfo(torch.int64).max
    if local_costs.numel() > 0:
        i = int(torch.argmin(local_costs).item())   # first minimum: lowest index
        mine = torch.tensor([int(local_costs[i].item()), first_plan + i], dtype=torch.int64)
    else:
        mine = torch.tensor([big, big], dtype=torch.int64)
    mine = mine.to(local_costs.device)
    if _group_size() > 1:
        parts = [torch.empty_like(mine) for _ in range(dist.get_world_size())]
        dist.all_gather(parts, mine)
    else:
        parts = [mine]
    best = min((int(p[0].item()), int(p[1].item())) for p in parts)
    return best
