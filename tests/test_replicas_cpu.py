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
