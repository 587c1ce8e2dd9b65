"""Host logic for runs over several GPUs (one process per GPU).

The single-mesh RHS is not sharded in this version: with N GPUs the benchmark runs N independent
replicas (weak scaling) and only reduces the step time. An ensemble of independent instances is
split across ranks with no collective at all: instances are assigned greedily by cost (largest
first, to the least-loaded rank), deterministically, so every rank computes the same assignment.
"""
from __future__ import annotations

from typing import Sequence


def assign_instances(costs: Sequence[float], world: int) -> list[list[int]]:
    """Greedy longest-processing-time assignment of instances to `world` ranks; returns, per rank,
    the ascending list of its instance indices. Ties go to the lower rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(dof: int, rhs_per_step: int, ms_per_step_max: float, world: int) -> float:
    """Whole-job GDOF.RHS/s of `world` replicas timed by the slowest rank."""
    return dof * rhs_per_step * world / (ms_per_step_max * 1e-3) / 1e9
