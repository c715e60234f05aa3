"""Sharding of independent work units across ranks (one process per GPU).

The simulator's workloads that span several GPUs are made of independent
units -- circuits of a batch, parameter sets of a gradient, repetitions of a
circuit -- so they are split across ranks with no collective on the data
path; the only collectives gather results and take the maximum time over
ranks for reporting.  ``torch.distributed`` provides the process group (NCCL
on GPUs, gloo on CPU).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def shard_range(n_units: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous balanced split: rank r gets [start, stop)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_by_cost(costs: Sequence[float], rank: int, world: int) -> List[int]:
    """Longest-processing-time assignment (deterministic): units sorted by
    decreasing cost go to the currently least loaded rank.  Returns the unit
    indices of `rank` in increasing order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    load = [0.0] * world
    mine = []
    for i in sorted(range(len(costs)), key=lambda j: (-costs[j], j)):
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += costs[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float (1 rank: the value itself)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(local: Sequence[float], indices: Sequence[int], total: int, device=None):
    """Scatter each rank's results into a length-`total` array on every rank."""
    import torch
    import torch.distributed as dist
    out = torch.zeros(total, dtype=torch.float64, device=device)
    out[torch.as_tensor(list(indices), dtype=torch.long, device=device)] = torch.as_tensor(
        list(local), dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(out, op=dist.ReduceOp.SUM)
    return out.cpu().numpy()
