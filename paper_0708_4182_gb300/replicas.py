"""Host-side logic of multi-GPU runs: one process per GPU, no data-path
collective.

The update shards naturally over independent domains (the channels of a
sweep) and over independent replicas of one domain. Each rank advances its
own share; the only collectives are a barrier and the reduction of timings
and counts for the report (torch.distributed, any backend: NCCL on GPUs,
gloo on the host for tests).
"""
from __future__ import annotations

import heapq


def partition(costs, rank: int, world: int) -> list:
    """Indices of the units (e.g. domains, cost = nodes) that ``rank`` of
    ``world`` owns: longest-processing-time-first assignment, each unit to
    the currently least loaded rank (ties to the lower rank), so every unit
    goes to exactly one rank and every rank computes the same split without
    communicating. Returned in ascending order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"bad rank {rank} of {world}")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0, r) for r in range(world)]
    owned = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            owned.append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return sorted(owned)


def loads(costs, world: int) -> list:
    """Total cost per rank under ``partition``."""
    return [sum(costs[i] for i in partition(costs, r, world)) for r in range(world)]


def _reduce(value: float, op, device) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    """Largest value over the ranks (the job's elapsed time is the slowest rank's)."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX, device)


def sum_over_ranks(value: float, device="cpu") -> float:
    """Sum over the ranks (units processed by the whole job)."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM, device)


def job_throughput(units: float, elapsed_s: float, device="cpu") -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return sum_over_ranks(units, device) / max_over_ranks(elapsed_s, device)
