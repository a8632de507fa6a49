"""Host-side logic of multi-GPU runs: one process per GPU, no data-path collective.

The all-pairs matrix splits into independent units -- whole studies when
several share a tree, and otherwise whole replicas of a study (the benchmark's
weak scaling).  Each rank computes its own units; the only communication is
the timing reduction after the timed region (max of the ranks' times, sum of
their units).  Nothing in the UniFrac arithmetic is exchanged between GPUs.
"""
from __future__ import annotations

from typing import Sequence


def shard_studies(sizes: Sequence[int], rank: int, world: int) -> list[int]:
    """Studies of `rank`: greedy longest-first assignment by pair count
    C(n, 2), ties broken by study index, so every study goes to exactly one
    rank and the ranks' pair counts are balanced."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    order = sorted(range(len(sizes)), key=lambda s: (-(sizes[s] * (sizes[s] - 1) // 2), s))
    load = [0] * world
    owner = [0] * len(sizes)
    for s in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[s] = r
        load[r] += sizes[s] * (sizes[s] - 1) // 2
    return [s for s in range(len(sizes)) if owner[s] == rank]


def reduce_timing(total_ms: float, units: float, dist=None, device=None) -> tuple[float, float]:
    """(max over ranks of the timed milliseconds, sum over ranks of the units)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(total_ms), float(units)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
