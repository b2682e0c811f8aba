"""Host-side work partitioning for runs on several GPUs (one process per GPU).

The Hermite-leapfrog workloads here split into independent problems: the
shots of a batch, or one seeded problem per rank.  Ranks exchange no data
while stepping; they only agree on who runs what and reduce their timings.
"""
from __future__ import annotations


def shard_by_cost(costs, world: int) -> list[list[int]]:
    """Assign items (e.g. shots, cost = nodes) to `world` ranks, longest first onto the
    least-loaded rank (LPT).  Deterministic: ties go to the lower rank and to the lower
    item index.  Returns, per rank, the sorted item indices."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of a per-rank float over the process group (the rank's own value without one)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    """The sum of a per-rank float over the process group."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
