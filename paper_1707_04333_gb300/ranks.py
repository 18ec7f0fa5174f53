"""Host-side logic for running the step on several GPUs, one process per GPU.

Independent instances need no exchange during a run, so ranks share nothing on
the data path: the batched form splits its instances across ranks, a single
instance runs as a replica per rank.  The only collectives are the reductions
of the timing and of the counts at the end, which work on CPU tensors (gloo)
as on device tensors (NCCL).
"""
from __future__ import annotations

from typing import Sequence


def shard_instances(costs: Sequence[float], world: int) -> list:
    """Split instances with estimated costs over `world` ranks by the greedy longest-processing-time
    rule: take instances in decreasing cost (ties: lower index first) and give each to the rank with
    the least load so far (ties: lower rank).  Returns, per rank, the ascending instance indices.
    Every instance lands on exactly one rank; no rank exceeds the mean load by more than the largest
    single cost."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def instance_cost(n_particles: int, n_triangles: int, per_triangle: float = 2.0) -> float:
    """Estimated step cost of one instance in particle-step units: its particles plus the field
    update, about two particle-steps' worth of memory traffic per triangle."""
    return float(n_particles) + per_triangle * float(n_triangles)


def _reduce(value: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (every rank gets it); the value itself without a process group."""
    return _reduce(value, "max", device)


def sum_over_ranks(value: float, device=None) -> float:
    """Sum over all ranks (every rank gets it); the value itself without a process group."""
    return _reduce(value, "sum", device)


def aggregate_rate(units_all_ranks: float, steps: int, ms_max: float) -> float:
    """Whole-job throughput: the units all ranks advanced per step times the steps, over the
    slowest rank's time."""
    return units_all_ranks * steps / (ms_max / 1e3)
