"""Multi-process host logic of multi-GPU runs, on CPU with the gloo backend:
study sharding covers every study exactly once with balanced pair counts,
and the timing reduction takes the slowest rank and the total units."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2107_05397_b300 import replicas


def test_shard_studies_partition_and_balance():
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in np.rint(np.exp(rng.uniform(np.log(200), np.log(6000), 64)))]
    for world in (1, 2, 3, 8):
        parts = [replicas.shard_studies(sizes, r, world) for r in range(world)]
        flat = sorted(s for p in parts for s in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[s] * (sizes[s] - 1) // 2 for s in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes) ** 2 / 2
    with pytest.raises(ValueError):
        replicas.shard_studies(sizes, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [300, 5000, 1200, 40, 2600, 900]
    mine = replicas.shard_studies(sizes, rank, world)
    units = float(sum(sizes[s] * (sizes[s] - 1) // 2 for s in mine))
    t, u = replicas.reduce_timing(10.0 + rank, units, dist, device="cpu")
    q.put((rank, mine, t, u))
    dist.destroy_process_group()


def test_gloo_two_ranks_timing_reduction():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = [300, 5000, 1200, 40, 2600, 900]
    total = float(sum(n * (n - 1) // 2 for n in sizes))
    studies = sorted(s for _, mine, _, _ in res for s in mine)
    assert studies == list(range(len(sizes)))
    for _, _, t, u in res:
        assert t == 11.0
        assert u == total


@pytest.mark.parametrize("n", [2, 3, 4, 9, 10, 257, 1000, 50000])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_stripes_partition_every_pair_once(n, world):
    """The ranks' stripe ranges are contiguous, cover every stripe, and their
    pairs (each stripe element as an unordered pair) cover every unordered
    pair exactly once across ranks, with pair counts within one stripe."""
    ranges = [replicas.shard_stripes(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == replicas.n_stripes(n)
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0 and a0 <= a1
    counts = [sum(replicas.stripe_pairs(n, s) for s in range(s0, s1)) for s0, s1 in ranges]
    assert sum(counts) == n * (n - 1) // 2
    assert max(counts) - min(counts) <= n
    if n > 1000:
        return
    owner = np.full((n, n), -1)
    for r, (s0, s1) in enumerate(ranges):
        i, j = replicas.stripe_pair_index(n, s0, s1)
        a, b = np.minimum(i, j), np.maximum(i, j)
        assert np.all(a < b)
        # a pair seen on two ranks would already have an owner
        prev = owner[a, b]
        assert np.all((prev == -1) | (prev == r))
        owner[a, b] = r
    iu = np.triu_indices(n, 1)
    assert np.all(owner[iu] >= 0)


def _stripe_worker(rank, world, port, n, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(9)
    D = rng.random((n, n))
    D = np.triu(D, 1) + np.triu(D, 1).T  # a symmetric matrix with a zero diagonal
    s0, s1 = replicas.shard_stripes(n, rank, world)
    i, j = replicas.stripe_pair_index(n, s0, s1)
    block = D[i, j].reshape(s1 - s0, n)  # what this rank's stripe range holds
    full = replicas.gather_condensed(block, n, dist)
    q.put((rank, (s0, s1), full))
    dist.destroy_process_group()


@pytest.mark.parametrize("n", [10, 11])
def test_gloo_two_ranks_stripe_gather_merges_the_matrix(n):
    """Two ranks each hold the stripe block of their range; the all-gather and
    host merge give every rank the whole condensed matrix."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stripe_worker, args=(r, world, port, n, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(9)
    D = rng.random((n, n))
    D = np.triu(D, 1) + np.triu(D, 1).T
    want = D[np.triu_indices(n, 1)]
    ranges = sorted(r for _, r, _ in res)
    assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == n // 2
    for _, _, full in res:
        np.testing.assert_array_equal(full, want)
