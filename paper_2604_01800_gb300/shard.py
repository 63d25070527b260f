"""Sharding of independent PPE systems across ranks (one process per GPU).

Independent systems need no data exchange: every rank solves its own share,
and the ranks meet only to agree on timings and to collect reports.  The
helpers work with any torch.distributed backend (NCCL between GPUs, gloo on
CPU for the tests); with no process group they reduce to the single-rank case.
"""
from __future__ import annotations

import heapq


def system_cost(nx: int, ny: int) -> float:
    """Estimated relative cost of one Jacobi-PCG solve of an nx x ny system:
    cells times iterations, the iterations growing like the grid's diameter."""
    return float(nx) * ny * max(nx, ny)


def partition(costs, world: int) -> list[list[int]]:
    """Greedy longest-processing-time partition of the systems (indices into
    `costs`) over `world` ranks: systems in decreasing cost, each to the rank
    with the least total so far (ties to the lower rank).  Deterministic, so
    every rank computes the same partition without communicating."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return [sorted(p) for p in parts]


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the slowest rank sets a job's
    time).  `device`: where the reduction tensor lives (a CUDA device for
    NCCL, None or 'cpu' for gloo)."""
    import torch
    dist = _dist()
    if dist is None:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_to_rank0(obj):
    """Every rank's `obj` as a list on rank 0 (rank order), None elsewhere."""
    dist = _dist()
    if dist is None:
        return [obj]
    rank, world = dist.get_rank(), dist.get_world_size()
    out = [None] * world if rank == 0 else None
    dist.gather_object(obj, out, dst=0)
    return out


def job_rate(units_per_rank, seconds_per_rank) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return float(sum(units_per_rank)) / max(seconds_per_rank)
