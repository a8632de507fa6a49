"""GPU parity on the three large workloads, through the C ABI, against the
FP64 oracle on seeded samples of their outputs.

* 50,000 samples on the 200,000-tip tree (about 400k kept branches): both
  variants in one mixed-precision call into the full 50,000 x 50,000 FP32
  layout (2 x 10 GB on the device), seeded rows against the oracle, every
  value in [0, 1], the rows equal to the matching columns.
* 64 studies of 200 to 6,000 samples sharing a 50,000-tip tree, all in one
  batched mixed-precision call: seeded rows of the largest study and the
  whole matrix of a study of fewer than 300 samples against the oracle.
* 25,000 samples on the 200,000-tip tree in FP64: one stripe range of both
  variants, a few hundred seeded pairs of it against the oracle at 1e-12.

Tolerances are those of every other parity test: 1e-12 (FP64) and 2e-6
(mixed precision), max abs over the compared elements.
"""
import numpy as np
import pytest

import oracle
from paper_2107_05397_b300 import binding as ub
from paper_2107_05397_b300 import synth

pytestmark = pytest.mark.gpu

TOL = {ub.FP64: 1e-12, ub.MIXED: 2e-6}
VARIANTS = [ub.UNWEIGHTED, ub.WEIGHTED_NORMALIZED]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ub.load()


def _sub_table(table, lo, hi):
    """Columns [lo, hi) of a table as a table of their own (renumbered)."""
    rows = np.repeat(np.arange(table.n_features), np.diff(table.indptr))
    m = (table.indices >= lo) & (table.indices < hi)
    return synth.coo_to_table(table.n_features, hi - lo, rows[m], table.indices[m] - lo,
                              table.counts[m], table.feature_node)


def _condensed_row(block, n, i):
    """Row i of a condensed block of n samples as a length-n vector (d(i, i) = 0)."""
    j = np.arange(n)
    a, b = np.minimum(i, j), np.maximum(i, j)
    idx = a * n - a * (a + 1) // 2 + (b - a - 1)
    return np.where(i == j, 0.0, block[np.where(i == j, 0, idx)])


# ------------------------------------------------------------------ 50,000 samples

def test_fifty_thousand_samples_full_layout_sampled_rows():
    """Both variants of 50,000 samples in one mixed-precision call, full FP32
    layout; four seeded rows of each against the oracle."""
    import torch
    w = synth.make_workload("tips200000_samples50000")
    N = w.table.n_samples
    rows = np.sort(np.random.default_rng(2024).choice(N, size=4, replace=False))
    got = {}
    with ub.Context(w.tree, w.table) as ctx:
        nb = ctx.output_bytes(ub.MIXED, ub.OUT_FULL)
        assert nb == 4 * N * N
        out = torch.empty(2 * N * N, dtype=torch.float32, device="cuda")
        ctx.run(ub.BOTH, ub.MIXED, ub.OUT_FULL, out=out)
        torch.cuda.synchronize()
        assert ctx.stat(ub.STAT_DEVICE_ERROR) == 0
        for v in VARIANTS:
            M = out[v * N * N:(v + 1) * N * N].view(N, N)
            assert float(M.min()) >= 0.0 and float(M.max()) <= 1.0
            r_t = torch.from_numpy(rows).cuda()
            rows_v = M.index_select(0, r_t)
            cols_v = M.index_select(1, r_t).t()
            assert torch.equal(rows_v, cols_v)  # symmetric on the sampled rows
            assert torch.all(rows_v[torch.arange(len(rows)), r_t] == 0)
            got[v] = rows_v.double().cpu().numpy()
        del out
        torch.cuda.empty_cache()
    for v in VARIANTS:
        ref, _ = oracle.unifrac_rows(w.tree, w.table, v, rows)
        err = float(np.max(np.abs(got[v] - ref)))
        assert err <= TOL[ub.MIXED], f"variant {v}: max abs err {err:.3e}"


# ------------------------------------------------------------------ 64 studies

def test_sixty_four_studies_largest_and_small_study():
    """The batched workload in one call (both variants, condensed blocks per
    study): four seeded rows of the largest study and the whole matrix of a
    study under 300 samples against the oracle."""
    import torch
    w = synth.make_workload("tips50000_studies64")
    offs = w.table.study_offsets
    sizes = np.diff(offs).astype(np.int64)
    assert len(sizes) == 64
    cond = sizes * (sizes - 1) // 2
    starts = np.concatenate([[0], np.cumsum(cond)])
    big = int(np.argmax(sizes))
    small_ids = [s for s in range(64) if 2 <= sizes[s] < 300]
    assert small_ids, "the seeded study sizes include one under 300 samples"
    small = small_ids[0]
    with ub.Context(w.tree, w.table) as ctx:
        nb = ctx.output_bytes(ub.MIXED, ub.OUT_CONDENSED)
        assert nb == 4 * int(cond.sum())
        out = ctx.run(ub.BOTH, ub.MIXED, ub.OUT_CONDENSED)
        torch.cuda.synchronize()
        assert ctx.stat(ub.STAT_DEVICE_ERROR) == 0
        host = out.cpu().numpy().astype(np.float64)
        del out
    total = int(cond.sum())
    assert host.min() >= 0.0 and host.max() <= 1.0
    for v in VARIANTS:
        vec = host[v * total:(v + 1) * total]
        # largest study: seeded rows
        n = int(sizes[big])
        sub = _sub_table(w.table, int(offs[big]), int(offs[big + 1]))
        blk = vec[starts[big]:starts[big + 1]]
        rows = np.sort(np.random.default_rng(31 + v).choice(n, size=4, replace=False))
        ref, _ = oracle.unifrac_rows(w.tree, sub, v, rows)
        for r, i in enumerate(rows):
            err = float(np.max(np.abs(_condensed_row(blk, n, i) - ref[r])))
            assert err <= TOL[ub.MIXED], f"study {big} row {i}: {err:.3e}"
        # a small study: every pair
        n = int(sizes[small])
        sub = _sub_table(w.table, int(offs[small]), int(offs[small + 1]))
        blk = vec[starts[small]:starts[small + 1]]
        ref = oracle.unifrac_full(w.tree, sub, v)
        iu = np.triu_indices(n, 1)
        err = float(np.max(np.abs(blk - ref[iu])))
        assert err <= TOL[ub.MIXED], f"study {small} ({n} samples): {err:.3e}"


# ------------------------------------------------------------------ 25,000 samples, FP64

@pytest.mark.parametrize("variant", VARIANTS)
def test_twenty_five_thousand_samples_fp64_stripe_range(variant):
    """FP64 mode on 25,000 samples: stripes [5000, 5064) (stripe s holds
    d(k, (k + s + 1) mod N)), 300 seeded elements against the oracle's
    per-pair distances at 1e-12."""
    import torch
    w = synth.make_workload("tips200000_samples25000")
    N = w.table.n_samples
    s0, s1 = 5000, 5064
    with ub.Context(w.tree, w.table) as ctx:
        assert ctx.n_stripes() == (N - 1 + 1) // 2
        out = ctx.run(variant, ub.FP64, ub.OUT_STRIPES, s0, s1)
        torch.cuda.synchronize()
        assert ctx.stat(ub.STAT_DEVICE_ERROR) == 0
        got = out.cpu().numpy().reshape(s1 - s0, N)
    assert got.min() >= 0.0 and got.max() <= 1.0
    rng = np.random.default_rng(77 + variant)
    s = rng.integers(0, s1 - s0, size=300)
    k = rng.integers(0, N, size=300)
    j = (k + s0 + s + 1) % N
    ref = oracle.unifrac_pairs(w.tree, w.table, variant, k, j)
    err = float(np.max(np.abs(got[s, k] - ref)))
    assert err <= TOL[ub.FP64], f"max abs err {err:.3e}"
