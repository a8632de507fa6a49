"""Host-side logic of multi-GPU runs: one process per GPU, no collective in
the UniFrac arithmetic.

The all-pairs matrix splits into independent units (Section II of the paper:
it is computed as a set of stripes that are merged afterwards):

* several studies on one tree: whole studies (`shard_studies`);
* one study: contiguous stripe ranges with equal pair counts
  (`shard_stripes`).  Stripe s holds d(k, (k + s + 1) mod n) for k in
  [0, n); every unordered pair lies in exactly one stripe, so disjoint stripe
  ranges hold disjoint pairs.  Each rank builds the whole embedding (cheap:
  O(branches x samples)) and runs the pair kernels of its range only
  (`unifrac_run` with that stripe range); the ranges are merged afterwards
  on the host (`stripes_to_condensed`), after an all-gather of the stripe
  blocks where every rank wants the whole matrix (`gather_condensed`).

The only communication besides that gather is the timing reduction after the
timed region (max of the ranks' times, sum of their units).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


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


def n_stripes(n: int) -> int:
    """ceil((n - 1) / 2): stripes of a study of n samples."""
    return n // 2 if n > 1 else 0


def stripe_pairs(n: int, s: int) -> int:
    """Distinct unordered pairs of stripe s: n, except the last stripe of an
    even n, whose elements k and k + n/2 are the same pair (n / 2 pairs)."""
    if n % 2 == 0 and s == n // 2 - 1:
        return n // 2
    return n


def shard_stripes(n: int, rank: int, world: int) -> tuple[int, int]:
    """Stripe range [s0, s1) of `rank` for one study of n samples: contiguous
    ranges in rank order whose pair counts differ by at most one stripe's n
    pairs (rank r starts at the stripe boundary nearest to r / world of the
    n (n - 1) / 2 pairs)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    S = n_stripes(n)
    total = n * (n - 1) // 2

    def start(r: int) -> int:
        if r >= world:
            return S
        # every stripe before the last holds n pairs: the start is the stripe
        # boundary nearest to r / world of the pairs
        target = r * total  # pairs before the start, times world
        return min(S, (2 * target + world * n) // (2 * world * n)) if n > 0 else 0

    return start(rank), start(rank + 1)


def stripe_pair_index(n: int, s0: int, s1: int) -> tuple[np.ndarray, np.ndarray]:
    """(i, j) of every element of the stripe block [s0, s1) x n, row-major:
    element (s, k) is d(k, (k + s0 + s + 1) mod n)."""
    s = np.arange(s0, s1, dtype=np.int64)[:, None]
    k = np.arange(n, dtype=np.int64)[None, :]
    i = np.broadcast_to(k, (s1 - s0, n))
    j = (k + s + 1) % n
    return i.reshape(-1), j.reshape(-1)


def stripes_to_condensed(block: np.ndarray, s0: int, s1: int, n: int,
                         out: np.ndarray) -> None:
    """Writes the stripe block [s0, s1) x n (row-major, as unifrac_run returns
    for UNIFRAC_OUT_STRIPES) into the condensed upper triangle `out`
    (n (n - 1) / 2, row-major i < j).  Only that range's pairs are written."""
    block = np.asarray(block).reshape(s1 - s0, n)
    i, j = stripe_pair_index(n, s0, s1)
    a, b = np.minimum(i, j), np.maximum(i, j)
    idx = a * n - a * (a + 1) // 2 + (b - a - 1)
    out[idx] = block.reshape(-1)


def gather_condensed(block: np.ndarray, n: int, dist, group=None) -> np.ndarray:
    """All-gather of the ranks' stripe blocks (each rank's range from
    `shard_stripes`) and host merge: the whole condensed matrix on every rank.
    `block` is this rank's [s1 - s0, n] stripe block on the host; blocks
    travel as float64 tensors over the process group's backend."""
    import torch
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    ranges = [shard_stripes(n, r, world) for r in range(world)]
    width = max((s1 - s0 for s0, s1 in ranges), default=0)
    s0, s1 = ranges[rank]
    mine = torch.zeros((width, n), dtype=torch.float64)
    mine[:s1 - s0] = torch.from_numpy(np.asarray(block, dtype=np.float64).reshape(s1 - s0, n))
    bufs = [torch.zeros((width, n), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    out = np.zeros(n * (n - 1) // 2, dtype=np.float64)
    for (r0, r1), b in zip(ranges, bufs):
        stripes_to_condensed(b[:r1 - r0].numpy(), r0, r1, n, out)
    return out


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
