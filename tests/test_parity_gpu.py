"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (max abs over every compared element): 1e-12 in FP64 mode and
2e-6 in mixed mode, the bounds the library documents for its two precisions.
"""
import numpy as np
import pytest

import oracle
from paper_2107_05397_b300 import binding as ub
from paper_2107_05397_b300 import synth

pytestmark = pytest.mark.gpu

TOL = {ub.FP64: 1e-12, ub.MIXED: 2e-6}
VARIANTS = [ub.UNWEIGHTED, ub.WEIGHTED_NORMALIZED]
PRECISIONS = [ub.FP64, ub.MIXED]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ub.load()


def run(tree, table, variant, precision, layout=ub.OUT_FULL, s0=0, s1=-1, host=False,
        options=None):
    import torch
    with ub.Context(tree, table) as ctx:
        for k, v in (options or {}).items():
            ctx.set_option(k, v)
        if host:  # True: pageable host memory; "pinned": page-locked
            nbytes = ctx.output_bytes(precision, layout, s0, s1) * (2 if variant == ub.BOTH else 1)
            dt = np.float64 if precision == ub.FP64 else np.float32
            n = nbytes // (8 if precision == ub.FP64 else 4)
            if host == "pinned":
                out = torch.zeros(n, dtype=torch.float64 if dt is np.float64 else torch.float32,
                                  pin_memory=True).numpy()
            else:
                out = np.zeros(n, dt)
            ctx.run(variant, precision, layout, s0, s1, out=out)
            return out.astype(np.float64)
        out = ctx.run(variant, precision, layout, s0, s1)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)


def condensed_to_full(c, n):
    m = np.zeros((n, n))
    iu = np.triu_indices(n, 1)
    m[iu] = c
    return m + m.T


def check_full(got, ref, precision):
    err = np.max(np.abs(got - ref)) if ref.size else 0.0
    assert err <= TOL[precision], f"max abs err {err:.3e}"
    return err


# ------------------------------------------------------------------ small workload

@pytest.fixture(scope="module")
def small():
    w = synth.make_workload("tips1024_samples256")
    ref = {v: oracle.unifrac_full(w.tree, w.table, v) for v in VARIANTS}
    return w, ref


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_small_workload_full_matrix(small, variant, precision):
    w, ref = small
    N = w.table.n_samples
    got = run(w.tree, w.table, variant, precision).reshape(N, N)
    check_full(got, ref[variant], precision)
    assert np.all(np.diag(got) == 0)
    np.testing.assert_array_equal(got, got.T)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_small_workload_condensed_and_host_output(small, variant, precision):
    w, ref = small
    N = w.table.n_samples
    dev = run(w.tree, w.table, variant, precision, ub.OUT_CONDENSED)
    host = run(w.tree, w.table, variant, precision, ub.OUT_CONDENSED, host=True)
    np.testing.assert_array_equal(dev, host)
    check_full(condensed_to_full(dev, N), ref[variant], precision)


# ------------------------------------------------------------------ ragged shapes

CASES = [
    # (seed, tips, samples, general tree, empty samples)
    (1, 6, 1, False, 0),
    (2, 6, 2, False, 0),
    (3, 9, 3, True, 0),
    (4, 40, 127, False, 3),
    (5, 40, 128, True, 0),
    (6, 64, 129, False, 2),
    (7, 300, 300, True, 5),
    (8, 200, 257, False, 0),
]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[2]}{'g' if c[3] else ''}" for c in CASES])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_ragged_random_cases(case, variant, precision):
    seed, tips, N, general, empty = case
    rng = np.random.default_rng(seed)
    tree, table = synth.random_case(rng, tips, N, density=0.2, general=general,
                                    empty_samples=empty)
    if general:  # zero-length branches too
        tree.length[rng.random(tree.n_nodes) < 0.1] = 0.0
        tree.length[-1] = 0.0
    ref = oracle.unifrac_full(tree, table, variant)
    got = run(tree, table, variant, precision).reshape(N, N)
    check_full(got, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_deep_caterpillar_tree(variant, precision):
    """A caterpillar (every internal node has one tip child): depth = tips."""
    n_tips = 400
    parent = []
    # postorder: tip0, tip1, int(0,1), tip2, int, tip3, int, ...
    nodes = 2 * n_tips - 1
    parent = np.full(nodes, -1, np.int32)
    parent[0] = 2
    parent[1] = 2
    cur = 2
    for t in range(2, n_tips):
        tip = 2 * t - 1
        new = 2 * t
        parent[cur] = new
        parent[tip] = new
        cur = new
    rng = np.random.default_rng(9)
    length = rng.exponential(0.2, nodes)
    length[-1] = 0.0
    tree = synth.Tree(parent=parent, length=length)
    tips = tree.tips()
    dense = (rng.random((tips.shape[0], 150)) < 0.05) * rng.integers(1, 9, (tips.shape[0], 150))
    table = synth.dense_to_table(dense, tips)
    ref = oracle.unifrac_full(tree, table, variant)
    got = run(tree, table, variant, precision).reshape(150, 150)
    check_full(got, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_common_features_span_several_tip_chunks(variant, precision):
    """Table rows longer than the embedding's 256-entry row chunks: features
    present in every sample, in 90 % and in 60 % of them (chunk ends inside
    128-column tiles, so two chunks share a tile), beside sparse ones."""
    rng = np.random.default_rng(31)
    tree = synth.yule_tree(300, rng, 0.1)
    tips = tree.tips()
    N = 700
    dense = (rng.random((tips.shape[0], N)) < 0.03) * rng.integers(1, 20, (tips.shape[0], N))
    for f, p in ((0, 1.0), (1, 0.9), (2, 0.9), (3, 0.6), (40, 1.0)):
        dense[f] = (rng.random(N) < p) * rng.integers(1, 50, N)
    table = synth.dense_to_table(dense, tips)
    ref = oracle.unifrac_full(tree, table, variant)
    got = run(tree, table, variant, precision).reshape(N, N)
    check_full(got, ref, precision)


def test_star_tree_disjoint_samples_unweighted_is_one():
    F, N = 200, 64
    tree = synth.star_tree(F, 0.25)
    dense = np.zeros((F, N), np.int64)
    for i in range(N):  # disjoint feature blocks
        dense[3 * i:3 * i + 3, i] = i + 1
    table = synth.dense_to_table(dense, np.arange(F, dtype=np.int32))
    for p in PRECISIONS:
        got = run(tree, table, ub.UNWEIGHTED, p).reshape(N, N)
        off = got[~np.eye(N, dtype=bool)]
        assert np.all(np.abs(off - 1.0) <= TOL[p])


# ------------------------------------------------------------------ layouts / stripes

@pytest.mark.parametrize("N", [130, 131])
@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_stripes_layout_and_merge(N, variant, precision):
    rng = np.random.default_rng(100 + N)
    tree, table = synth.random_case(rng, 120, N, density=0.15)
    ref = oracle.unifrac_full(tree, table, variant)
    nst = N // 2
    st = run(tree, table, variant, precision, ub.OUT_STRIPES, 0, -1).reshape(nst, N)
    k = np.arange(N)
    for s in range(nst):
        exp = ref[k, (k + s + 1) % N]
        assert np.max(np.abs(st[s] - exp)) <= TOL[precision]
    # partial stripe range
    part = run(tree, table, variant, precision, ub.OUT_STRIPES, 3, 17).reshape(14, N)
    np.testing.assert_array_equal(part, st[3:17])
    # condensed runs over disjoint stripe ranges merge into the whole
    import torch
    dt = torch.float64 if precision == ub.FP64 else torch.float32
    with ub.Context(tree, table) as ctx:
        nb = ctx.output_bytes(precision, ub.OUT_CONDENSED)
        buf = torch.full((nb // (8 if precision == ub.FP64 else 4),), -7.0, dtype=dt, device="cuda")
        a = nst // 3
        ctx.run(variant, precision, ub.OUT_CONDENSED, 0, a, out=buf)
        touched = buf.cpu().numpy() != -7.0
        assert 0 < touched.sum() < buf.numel()
        ctx.run(variant, precision, ub.OUT_CONDENSED, a, nst, out=buf)
        merged = buf.cpu().numpy().astype(np.float64)
        whole = ctx.run(variant, precision, ub.OUT_CONDENSED).cpu().numpy().astype(np.float64)
        np.testing.assert_array_equal(merged, whole)
        full = torch.full((N * N,), -7.0, dtype=dt, device="cuda")
        ctx.run(variant, precision, ub.OUT_FULL, 0, a, out=full)
        ctx.run(variant, precision, ub.OUT_FULL, a, nst, out=full)
        np.testing.assert_array_equal(condensed_to_full(whole, N),
                                      full.cpu().numpy().astype(np.float64).reshape(N, N))


# ------------------------------------------------------------------ studies

@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("layout", [ub.OUT_CONDENSED, ub.OUT_FULL])
def test_several_studies(variant, precision, layout):
    rng = np.random.default_rng(55)
    tree = synth.yule_tree(500, rng, 0.1)
    sizes = [130, 0, 1, 2, 257, 40]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    N = int(offs[-1])
    tips = tree.tips()
    dense = (rng.random((tips.shape[0], N)) < 0.03) * rng.integers(1, 30, (tips.shape[0], N))
    table = synth.dense_to_table(dense, tips)
    table.study_offsets = offs
    got = run(tree, table, variant, precision, layout)
    pos = 0
    for s, n in enumerate(sizes):
        sub = synth.dense_to_table(dense[:, offs[s]:offs[s + 1]], tips)
        ref = oracle.unifrac_full(tree, sub, variant) if n else np.zeros((0, 0))
        if layout == ub.OUT_FULL:
            blk = got[pos:pos + n * n].reshape(n, n)
            pos += n * n
        else:
            blk = condensed_to_full(got[pos:pos + n * (n - 1) // 2], n)
            pos += n * (n - 1) // 2
        check_full(blk, ref, precision)
    assert pos == got.shape[0]


# ------------------------------------------------------------------ full-size workload

@pytest.fixture(scope="module")
def large():
    return synth.make_workload("tips32768_samples4096")


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_large_workload_sampled_rows(large, variant, precision):
    """Full condensed run on 4,096 samples; sampled rows against the oracle."""
    w = large
    N = w.table.n_samples
    got = run(w.tree, w.table, variant, precision, ub.OUT_CONDENSED)
    assert got.shape[0] == N * (N - 1) // 2
    assert got.min() >= 0.0 and got.max() <= 1.0
    rows = np.random.default_rng(3).choice(N, size=4, replace=False)
    ref, _ = oracle.unifrac_rows(w.tree, w.table, variant, rows)
    for r, i in enumerate(rows):
        j = np.arange(N)
        a, b = np.minimum(i, j), np.maximum(i, j)
        idx = a * N - a * (a + 1) // 2 + (b - a - 1)
        vals = np.where(i == j, 0.0, got[np.where(i == j, 0, idx)])
        assert np.max(np.abs(vals - ref[r])) <= TOL[precision]


@pytest.mark.parametrize("layout", [ub.OUT_FULL, ub.OUT_CONDENSED])
def test_host_copy_ranges_ragged_matrix(layout):
    """Row-range host copies of a matrix whose last tile is partial (1,700
    samples: 14 tiles, two block rows of the work list): bit-identical to a
    device-memory run for 1, 2, 5 and 64 ranges, equal to the oracle."""
    import torch
    rng = np.random.default_rng(1700)
    tree, table = synth.random_case(rng, 200, 1700, density=0.04, general=True,
                                    empty_samples=3)
    N = table.n_samples
    ref = {v: oracle.unifrac_full(tree, table, v) for v in VARIANTS}
    with ub.Context(tree, table) as ctx:
        dev = ctx.run(ub.BOTH, ub.MIXED, layout)
        torch.cuda.synchronize()
        dev = dev.cpu().numpy()
        for ranges in (1, 2, 5, 64):
            ctx.set_option(ub.OPT_COPY_RANGES, ranges)
            host = torch.full((dev.size,), -1.0, dtype=torch.float32, pin_memory=True).numpy()
            ctx.run(ub.BOTH, ub.MIXED, layout, out=host)
            np.testing.assert_array_equal(host, dev)
    half = dev.size // 2
    for v, part in ((ub.UNWEIGHTED, dev[:half]), (ub.WEIGHTED_NORMALIZED, dev[half:])):
        got = part.reshape(N, N) if layout == ub.OUT_FULL else condensed_to_full(part, N)
        check_full(got.astype(np.float64), ref[v], ub.MIXED)


def test_device_block_cache_reuse_changes_nothing(large):
    """Contexts take the work buffers earlier contexts freed (the library's
    cache of device blocks, dirty) and give the same matrices bit for bit;
    the blocks are reused, not piled up; a cap of 0 turns the cache off and
    releasing it empties it."""
    import torch
    w = large
    ub.unifrac_release_cached_memory(-1)
    ub.unifrac_set_memory_cache(-1)
    assert ub.unifrac_cached_memory() == 0

    def one_run():
        with ub.Context(w.tree, w.table) as ctx:
            out = ctx.run(ub.BOTH, ub.MIXED, ub.OUT_CONDENSED)
            torch.cuda.synchronize()
            return out.cpu().numpy()

    cold = one_run()
    held = ub.unifrac_cached_memory()
    assert held >= 64 << 20  # the counts array alone is about 1 GB here
    for _ in range(2):
        np.testing.assert_array_equal(one_run(), cold)
        assert ub.unifrac_cached_memory() == held
    ub.unifrac_set_memory_cache(0)
    assert ub.unifrac_cached_memory() == 0
    np.testing.assert_array_equal(one_run(), cold)
    assert ub.unifrac_cached_memory() == 0
    ub.unifrac_set_memory_cache(-1)
    np.testing.assert_array_equal(one_run(), cold)
    assert ub.unifrac_cached_memory() == held
    ub.unifrac_release_cached_memory(-1)
    assert ub.unifrac_cached_memory() == 0
    with pytest.raises(ub.UniFracError):
        ub.unifrac_set_memory_cache(-2)


@pytest.mark.parametrize("layout", [ub.OUT_FULL, ub.OUT_CONDENSED])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_host_copy_ranges_change_nothing(large, precision, layout):
    """Into pinned host memory the weighted matrix leaves in row ranges, each
    copied while the next computes (UNIFRAC_OPT_COPY_RANGES): 4,096 samples
    (32 tiles, three block rows) give several ranges; every range count gives
    the matrices of a device-memory run bit for bit, and sampled rows agree
    with the oracle."""
    import torch
    w = large
    N = w.table.n_samples
    with ub.Context(w.tree, w.table) as ctx:
        dev = ctx.run(ub.BOTH, precision, layout)
        torch.cuda.synchronize()
        dev = dev.cpu().numpy()
        dt = torch.float64 if precision == ub.FP64 else torch.float32
        for ranges in (1, 3, 8, 64):
            ctx.set_option(ub.OPT_COPY_RANGES, ranges)
            assert ctx.get_option(ub.OPT_COPY_RANGES) == ranges
            host = torch.full((dev.size,), -1.0, dtype=dt, pin_memory=True).numpy()
            ctx.run(ub.BOTH, precision, layout, out=host)
            np.testing.assert_array_equal(host, dev)
        with pytest.raises(ub.UniFracError):
            ctx.set_option(ub.OPT_COPY_RANGES, 0)
    half = dev.size // 2
    rows = np.array([5, N // 2 + 3, N - 1])
    for v, part in ((ub.UNWEIGHTED, dev[:half]), (ub.WEIGHTED_NORMALIZED, dev[half:])):
        ref, _ = oracle.unifrac_rows(w.tree, w.table, v, rows)
        for r, i in enumerate(rows):
            if layout == ub.OUT_FULL:
                vals = part.reshape(N, N)[i].astype(np.float64)
            else:
                j = np.arange(N)
                a, b = np.minimum(i, j), np.maximum(i, j)
                idx = a * N - a * (a + 1) // 2 + (b - a - 1)
                vals = np.where(i == j, 0.0, part[np.where(i == j, 0, idx)]).astype(np.float64)
            assert np.max(np.abs(vals - ref[r])) <= TOL[precision]


@pytest.mark.parametrize("threshold", [0, 1, 40, 10**9])
@pytest.mark.parametrize("case", [0, 1])
def test_weighted_dense_sparse_split(small, threshold, case):
    """Every dense / sparse split of the weighted mixed kernel (all dense, a
    split, all sparse) agrees with the oracle."""
    if case == 0:
        w, ref = small
        tree, table, r = w.tree, w.table, ref[ub.WEIGHTED_NORMALIZED]
    else:
        rng = np.random.default_rng(77)
        tree, table = synth.random_case(rng, 300, 261, density=0.05, general=True,
                                        empty_samples=2)
        r = oracle.unifrac_full(tree, table, ub.WEIGHTED_NORMALIZED)
    N = table.n_samples
    got = run(tree, table, ub.WEIGHTED_NORMALIZED, ub.MIXED,
              options={ub.OPT_SPARSE_THRESHOLD: threshold}).reshape(N, N)
    check_full(got, r, ub.MIXED)


@pytest.mark.parametrize("threshold", [0, 1, 40, 10**9])
@pytest.mark.parametrize("case", [0, 1])
def test_unweighted_tensor_sparse_split(small, threshold, case):
    """Every split of the unweighted tensor-core path (all tensor core, a
    split, everything but one K-tile sparse) agrees with the oracle."""
    if case == 0:
        w, ref = small
        tree, table, r = w.tree, w.table, ref[ub.UNWEIGHTED]
    else:
        rng = np.random.default_rng(78)
        tree, table = synth.random_case(rng, 300, 261, density=0.05, general=True,
                                        empty_samples=2)
        r = oracle.unifrac_full(tree, table, ub.UNWEIGHTED)
    N = table.n_samples
    got = run(tree, table, ub.UNWEIGHTED, ub.MIXED,
              options={ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD: threshold}).reshape(N, N)
    check_full(got, r, ub.MIXED)


def test_sparse_lane_bound_changes_nothing(small):
    """The sparse kernels' single-lane incidence bound only moves work between
    two paths that add the same exact integers: every bound gives bit-identical
    matrices (all positions sparse), equal to the oracle's within tolerance."""
    w, ref = small
    N = w.table.n_samples
    for variant, th_opt, lane_opt in (
            (ub.WEIGHTED_NORMALIZED, ub.OPT_SPARSE_THRESHOLD, ub.OPT_SPARSE_LANE_PAIRS),
            (ub.UNWEIGHTED, ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD,
             ub.OPT_UNWEIGHTED_SPARSE_LANE_PAIRS)):
        outs = []
        for lane in (0, 1, 16, 64, 4096):
            got = run(w.tree, w.table, variant, ub.MIXED,
                      options={th_opt: 10**9, lane_opt: lane}).reshape(N, N)
            check_full(got, ref[variant], ub.MIXED)
            outs.append(got)
        for o in outs[1:]:
            np.testing.assert_array_equal(o, outs[0])


@pytest.mark.parametrize("variant", VARIANTS)
def test_rare_branch_lists_ignore_dirty_device_memory(variant, small):
    """The list index counts only flagged (tile, position) cells: with the
    device memory the library's buffers come from first filled with 0xFF
    bytes and freed, every list bound still gives the oracle's matrix."""
    import torch
    th_opt, list_opt = ((ub.OPT_SPARSE_THRESHOLD, ub.OPT_RARE_LIST)
                        if variant == ub.WEIGHTED_NORMALIZED else
                        (ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD, ub.OPT_UNWEIGHTED_RARE_LIST))
    w, ref = small
    N = w.table.n_samples
    for bound in (12, 4096):
        torch.cuda.empty_cache()
        dirty = torch.full((1 << 28,), 255, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        del dirty
        torch.cuda.empty_cache()
        got = run(w.tree, w.table, variant, ub.MIXED,
                  options={th_opt: 10**9, list_opt: bound}).reshape(N, N)
        check_full(got, ref[variant], ub.MIXED)


@pytest.mark.parametrize("variant", VARIANTS)
def test_rare_branch_lists_change_nothing(variant, small):
    """Branches present in few samples summed from per-branch lists (every
    pair of their samples) instead of the sparse kernel's walk: the same exact
    integers, so bit-identical matrices for every list bound -- off, some,
    every sparse position listed -- on one study, several studies and a stripe
    range of a study; equal to the oracle within tolerance."""
    th_opt, list_opt = ((ub.OPT_SPARSE_THRESHOLD, ub.OPT_RARE_LIST)
                        if variant == ub.WEIGHTED_NORMALIZED else
                        (ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD, ub.OPT_UNWEIGHTED_RARE_LIST))
    w, ref = small
    N = w.table.n_samples
    outs = []
    for bound in (0, 3, 12, 4096):
        got = run(w.tree, w.table, variant, ub.MIXED,
                  options={th_opt: 10**9, list_opt: bound}).reshape(N, N)
        check_full(got, ref[variant], ub.MIXED)
        outs.append(got)
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    # the list phase's statistics: none listed at bound 0; with every sparse
    # position listed, the sparse kernel does nothing and the lists make
    # exactly the co-present pairs sum_b C(n_b, 2) of those positions -- all
    # kept branches weighted; all but the 64 most present unweighted (the
    # tensor cores always take one K-tile of 64 positions)
    P = _presence(w.tree, w.table)
    n = w.tree.n_nodes
    nb = P[:n - 1].sum(axis=1)
    nb = np.sort(nb[(nb > 0) & (w.tree.length[:n - 1] > 0)])[::-1].astype(np.float64)
    if variant == ub.UNWEIGHTED:
        nb = nb[64:]
    want = float(np.sum(nb * (nb - 1) / 2))
    lst, upd = ((ub.STAT_LIST_UPDATES_WEIGHTED, ub.STAT_SPARSE_UPDATES_WEIGHTED)
                if variant == ub.WEIGHTED_NORMALIZED else
                (ub.STAT_LIST_UPDATES_UNWEIGHTED, ub.STAT_SPARSE_UPDATES_UNWEIGHTED))
    for bound in (0, 4096):
        with ub.Context(w.tree, w.table) as ctx:
            ctx.set_option(th_opt, 10**9)
            ctx.set_option(list_opt, bound)
            ctx.run(variant, ub.MIXED, ub.OUT_CONDENSED)
            n_list, n_sparse = ctx.stat(lst), ctx.stat(upd)
            if bound == 0:
                assert n_list == 0 and n_sparse > 0
            else:
                assert n_sparse == 0 and n_list == want
    # several studies (pairs only within a study) and a stripe range
    rng = np.random.default_rng(58)
    tree = synth.yule_tree(700, rng, 0.1)
    sizes = [300, 5, 129, 0, 260, 1]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    tips = tree.tips()
    dense = (rng.random((tips.shape[0], int(offs[-1]))) < 0.04) * \
        rng.integers(1, 30, (tips.shape[0], int(offs[-1])))
    table = synth.dense_to_table(dense, tips)
    table.study_offsets = offs
    multi = [run(tree, table, variant, ub.MIXED, ub.OUT_CONDENSED,
                 options={th_opt: 40, list_opt: bound}) for bound in (0, 8, 4096)]
    for o in multi[1:]:
        np.testing.assert_array_equal(o, multi[0])
    one = synth.dense_to_table(dense[:, :300], tips)
    ref1 = oracle.unifrac_full(tree, one, variant)
    check_full(condensed_to_full(multi[1][:300 * 299 // 2], 300), ref1, ub.MIXED)
    stripes = [run(tree, one, variant, ub.MIXED, ub.OUT_STRIPES, 40, 77,
                   options={th_opt: 30, list_opt: bound}) for bound in (0, 8, 4096)]
    for o in stripes[1:]:
        np.testing.assert_array_equal(o, stripes[0])
    blk = stripes[1].reshape(77 - 40, 300)
    k = np.arange(300)
    for si, s_ in enumerate(range(40, 77)):
        np.testing.assert_allclose(blk[si], ref1[k, (k + s_ + 1) % 300], rtol=0, atol=2e-6)


@pytest.mark.parametrize("variant", VARIANTS)
def test_persistent_work_queue_equals_one_cta_per_item(variant):
    """Pair kernels pulling work items from a device queue (persistent grid)
    and one CTA per item compute each tile pair the same way: bit-identical
    matrices, several studies, dense and sparse parts both in use, and equal
    to the oracle within tolerance."""
    rng = np.random.default_rng(57)
    tree = synth.yule_tree(700, rng, 0.1)
    sizes = [300, 5, 129, 0, 260, 1]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    N = int(offs[-1])
    tips = tree.tips()
    dense = (rng.random((tips.shape[0], N)) < 0.04) * rng.integers(1, 30, (tips.shape[0], N))
    table = synth.dense_to_table(dense, tips)
    table.study_offsets = offs
    opts = {ub.OPT_SPARSE_THRESHOLD: 40, ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD: 20}
    outs = []
    for persistent in (0, 1):
        outs.append(run(tree, table, variant, ub.MIXED, ub.OUT_CONDENSED,
                        options={**opts, ub.OPT_PERSISTENT: persistent}))
    np.testing.assert_array_equal(outs[0], outs[1])
    pos = 0
    for s, n in enumerate(sizes):
        m = n * (n - 1) // 2
        if n > 1:
            sub = synth.dense_to_table(dense[:, offs[s]:offs[s + 1]], tips)
            ref = oracle.unifrac_full(tree, sub, variant)
            check_full(condensed_to_full(outs[1][pos:pos + m], n), ref, ub.MIXED)
        pos += m


@pytest.mark.parametrize("kernel", [1, 2])
def test_unweighted_mixed_kernel_choice(small, kernel):
    """Both unweighted mixed-precision kernels (tensor-core Gram, bit-packed
    lookup) agree with the oracle."""
    w, ref = small
    N = w.table.n_samples
    got = run(w.tree, w.table, ub.UNWEIGHTED, ub.MIXED,
              options={ub.OPT_UNWEIGHTED_MIXED_KERNEL: kernel}).reshape(N, N)
    check_full(got, ref[ub.UNWEIGHTED], ub.MIXED)


@pytest.mark.parametrize("variant", VARIANTS)
def test_graph_replay_matches_eager(small, variant):
    """With CUDA-graph replay on, the first run executes eagerly and captures;
    later identical runs replay the graph.  Results must be bit-identical, and
    a change of layout, option or output buffer must not replay a stale graph."""
    import torch
    w, ref = small
    N = w.table.n_samples
    with ub.Context(w.tree, w.table) as ctx:
        eager = ctx.run(variant, ub.MIXED, ub.OUT_CONDENSED).cpu().numpy()
        ctx.set_option(ub.OPT_USE_GRAPH, 1)
        out = torch.full((N * (N - 1) // 2,), -1.0, device="cuda")
        for rep in range(3):
            out.fill_(-1.0)
            ctx.run(variant, ub.MIXED, ub.OUT_CONDENSED, out=out)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), eager)
            # timing events recorded inside the replayed graph stay queryable
            stat = ub.STAT_PAIR_MS_UNWEIGHTED if variant == ub.UNWEIGHTED else ub.STAT_PAIR_MS_WEIGHTED
            assert ctx.stat(stat) > 0
            assert ctx.stat(ub.STAT_EMBED_MS) > 0
        full = ctx.run(variant, ub.MIXED, ub.OUT_FULL)
        full2 = ctx.run(variant, ub.MIXED, ub.OUT_FULL, out=full.clone().fill_(-1.0))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(full.cpu().numpy(), full2.cpu().numpy())
        check_full(full.cpu().numpy().reshape(N, N).astype(np.float64), ref[variant], ub.MIXED)
        other = 1 - variant
        o2 = ctx.run(other, ub.MIXED, ub.OUT_CONDENSED)
        check_full(condensed_to_full(o2.cpu().numpy().astype(np.float64), N), ref[other], ub.MIXED)
        ctx.set_option(ub.OPT_SPARSE_THRESHOLD, 7)
        o3 = ctx.run(variant, ub.MIXED, ub.OUT_CONDENSED, out=out)
        o3 = ctx.run(variant, ub.MIXED, ub.OUT_CONDENSED, out=out)
        torch.cuda.synchronize()
        check_full(condensed_to_full(o3.cpu().numpy().astype(np.float64), N), ref[variant], ub.MIXED)


def test_repeat_runs_bit_identical(small):
    w, _ = small
    for v in VARIANTS:
        for p in PRECISIONS:
            a = run(w.tree, w.table, v, p)
            b = run(w.tree, w.table, v, p)
            np.testing.assert_array_equal(a, b)


def test_run_argument_errors(small):
    import torch
    w, _ = small
    with ub.Context(w.tree, w.table) as ctx:
        small_buf = torch.zeros(10, dtype=torch.float32, device="cuda")
        with pytest.raises(ub.UniFracError) as ei:
            ctx.run(ub.UNWEIGHTED, ub.MIXED, ub.OUT_FULL, out=small_buf)
        assert ei.value.status == -5
        with pytest.raises(ub.UniFracError) as ei:
            ctx.run(ub.UNWEIGHTED, ub.MIXED, ub.OUT_STRIPES, 5, 3)
        assert ei.value.status == -4
        with pytest.raises(ub.UniFracError) as ei:
            ctx.run(ub.UNWEIGHTED, ub.MIXED, ub.OUT_STRIPES, 0, 10_000)
        assert ei.value.status == -4
        with pytest.raises(ub.UniFracError) as ei:
            ub.unifrac_run(ctx.handle, 7, ub.MIXED, 0, -1, ub.OUT_FULL,
                           torch.zeros(w.table.n_samples ** 2, device="cuda"))
        assert ei.value.status == -1


def test_autotune_and_cache(small, tmp_path):
    """The tuner picks one of its candidates, caches it, and the tuned context
    still matches the oracle; a second context reuses the cached setting."""
    import torch
    from paper_2107_05397_b300 import autotune
    w, ref = small
    N = w.table.n_samples
    cache = str(tmp_path / "tune.json")
    for variant in VARIANTS:
        with ub.Context(w.tree, w.table) as ctx:
            rec = autotune.tune(ctx, variant, ub.MIXED, cache_path=cache)
            assert rec["cached"] is False
            if variant == ub.WEIGHTED_NORMALIZED:
                assert rec["flush"] in (128, 256, 512)
                assert rec["lane_pairs"] == ctx.get_option(ub.OPT_SPARSE_LANE_PAIRS)
            got = ctx.run(variant, ub.MIXED, ub.OUT_FULL).cpu().numpy().astype(np.float64)
            check_full(got.reshape(N, N), ref[variant], ub.MIXED)
        with ub.Context(w.tree, w.table) as ctx:
            rec2 = autotune.tune(ctx, variant, ub.MIXED, cache_path=cache)
            assert rec2["cached"] is True


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("layout", [ub.OUT_CONDENSED, ub.OUT_FULL, ub.OUT_STRIPES])
def test_both_variants_in_one_run(small, precision, layout):
    """UNIFRAC_BOTH (one embedding pass) equals the two single-variant runs."""
    w, _ = small
    with ub.Context(w.tree, w.table) as ctx:
        both = ctx.run(ub.BOTH, precision, layout).cpu().numpy()
        uw = ctx.run(ub.UNWEIGHTED, precision, layout).cpu().numpy()
        wn = ctx.run(ub.WEIGHTED_NORMALIZED, precision, layout).cpu().numpy()
    np.testing.assert_array_equal(both, np.concatenate([uw, wn]))
    for kind in (True, "pinned"):  # pinned: the first result's copy overlaps the second
        host = run(w.tree, w.table, ub.BOTH, precision, layout, host=kind)
        np.testing.assert_array_equal(host, np.concatenate([uw, wn]).astype(np.float64))


@pytest.mark.parametrize("graph", [0, 1])
def test_both_overlapped_equals_serial(small, graph):
    """UNIFRAC_BOTH with the variants on two streams is bit-identical to the
    serial run (both variants with a sparse-kernel part -- per-branch lists
    off, or every sparse branch of these 256 samples would be listed -- eager
    and graph replay)."""
    import torch
    w, _ = small
    opts = {ub.OPT_SPARSE_THRESHOLD: 24, ub.OPT_UNWEIGHTED_SPARSE_THRESHOLD: 12,
            ub.OPT_RARE_LIST: 0, ub.OPT_UNWEIGHTED_RARE_LIST: 0}
    with ub.Context(w.tree, w.table) as ctx:
        for k, v in opts.items():
            ctx.set_option(k, v)
        ctx.set_option(ub.OPT_USE_GRAPH, graph)
        ctx.set_option(ub.OPT_OVERLAP_VARIANTS, 0)
        serial = ctx.run(ub.BOTH, ub.MIXED, ub.OUT_CONDENSED).cpu().numpy()
        ctx.set_option(ub.OPT_OVERLAP_VARIANTS, 1)
        assert ctx.get_option(ub.OPT_OVERLAP_VARIANTS) == 1
        for _ in range(3):
            over = ctx.run(ub.BOTH, ub.MIXED, ub.OUT_CONDENSED)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(over.cpu().numpy(), serial)
        assert ctx.stat(ub.STAT_DEVICE_ERROR) == 0
        assert ctx.stat(ub.STAT_SPARSE_UPDATES_WEIGHTED) > 0
        assert ctx.stat(ub.STAT_SPARSE_UPDATES_UNWEIGHTED) > 0
        assert ctx.stat(ub.STAT_SELECTED_WEIGHTED) > 0
        for sp, pair in ((ub.STAT_SPARSE_MS_WEIGHTED, ub.STAT_PAIR_MS_WEIGHTED),
                         (ub.STAT_SPARSE_MS_UNWEIGHTED, ub.STAT_PAIR_MS_UNWEIGHTED)):
            # the sparse kernel is timed inside its variant's pair phase
            assert 0.0 < ctx.stat(sp) <= ctx.stat(pair)
    for kind in (True, "pinned"):
        for overlap in (0, 1):
            host = run(w.tree, w.table, ub.BOTH, ub.MIXED, ub.OUT_CONDENSED, host=kind,
                       options={**opts, ub.OPT_OVERLAP_VARIANTS: overlap})
            np.testing.assert_array_equal(host, serial.astype(np.float64))


@pytest.mark.parametrize("variant", VARIANTS)
def test_paper_scale_workload_sampled_rows(variant):
    """25,000 samples on a 200,000-tip tree (EMP-sized; about 396k kept
    branches): one mixed-precision run of both variants, sampled rows
    against the oracle, and every value in [0, 1]."""
    import torch
    w = _paper_scale()
    N = w.table.n_samples
    with ub.Context(w.tree, w.table) as ctx:
        nb = ctx.output_bytes(ub.MIXED, ub.OUT_CONDENSED)
        out = ctx.run(ub.BOTH, ub.MIXED, ub.OUT_CONDENSED)
        torch.cuda.synchronize()
        got = out[variant * (nb // 4):(variant + 1) * (nb // 4)].cpu().numpy().astype(np.float64)
        del out
    assert got.min() >= 0.0 and got.max() <= 1.0
    rows = np.random.default_rng(11 + variant).choice(N, size=2, replace=False)
    ref, _ = oracle.unifrac_rows(w.tree, w.table, variant, rows)
    for r, i in enumerate(rows):
        j = np.arange(N)
        a, b = np.minimum(i, j), np.maximum(i, j)
        idx = a * N - a * (a + 1) // 2 + (b - a - 1)
        vals = np.where(i == j, 0.0, got[np.where(i == j, 0, idx)])
        assert np.max(np.abs(vals - ref[r])) <= TOL[ub.MIXED]


_PAPER_SCALE = []


def _paper_scale():
    if not _PAPER_SCALE:
        _PAPER_SCALE.append(synth.make_workload("tips200000_samples25000"))
    return _PAPER_SCALE[0]


# ------------------------------------------------------------------ create statistics

def _presence(tree, table):
    """[n_nodes, N] presence of every node in every sample, from the oracle."""
    return np.stack([oracle.embedding(tree, table, i)[1] for i in range(table.n_samples)],
                    axis=1).astype(bool)


def _expected_stats(tree, table, offs):
    P = _presence(tree, table)
    n = tree.parent.shape[0]
    root = n - 1
    eligible = (np.arange(n) < root) & (tree.length > 0)
    pair_branch = useful = 0.0
    for s in range(len(offs) - 1):
        sub = P[:, offs[s]:offs[s + 1]]
        ns = sub.shape[1]
        nb = sub.sum(axis=1)
        pair_branch += ns * (ns - 1) / 2 * int(np.count_nonzero(eligible & (nb > 0)))
        useful += float(np.sum(nb[eligible] * (nb[eligible] - 1) / 2))
    kept = int(np.count_nonzero(eligible & P.any(axis=1)))
    reach = int(P[:root].sum(axis=0).max()) if P.shape[1] else 0
    return pair_branch, useful, kept, reach


def test_create_statistics_several_studies():
    # pair x branch, co-present pairs and kept branches, per study, from the
    # oracle's presence embedding; zero-length branches and empty studies
    rng = np.random.default_rng(91)
    tree = synth.yule_tree(400, rng, 0.1)
    tree.length[rng.choice(tree.parent.shape[0] - 1, 40, replace=False)] = 0.0
    sizes = [130, 0, 1, 2, 200, 40]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    tips = tree.tips()
    dense = (rng.random((tips.shape[0], int(offs[-1]))) < 0.04) * \
        rng.integers(1, 30, (tips.shape[0], int(offs[-1])))
    table = synth.dense_to_table(dense, tips)
    table.study_offsets = offs
    pb, us, kept, reach = _expected_stats(tree, table, offs)
    with ub.Context(tree, table) as ctx:
        assert ctx.stat(ub.STAT_PAIR_BRANCH) == pb
        assert ctx.stat(ub.STAT_USEFUL) == us
        assert ctx.stat(ub.STAT_BRANCHES_KEPT) == kept
        assert ctx.stat(ub.STAT_MAX_REACH) >= reach  # small tree: the bound
        assert ctx.stat(ub.STAT_CREATE_HOST_MS) >= 0.0


def test_create_statistics_large_tree_exact_reach():
    # a tree with more than 65,793 branches: the reach is counted exactly
    # (bit-sliced column counters over several column blocks)
    rng = np.random.default_rng(92)
    tree = synth.yule_tree(34000, rng, 0.1)
    N = 1100  # 18 words of columns: more than one 8 MiB block of bitsets
    tips = tree.tips()
    dense = (rng.random((tips.shape[0], N)) < 0.01) * rng.integers(1, 9, (tips.shape[0], N))
    dense[:, 5] = 0  # an empty sample
    table = synth.dense_to_table(dense, tips)
    pb, us, kept, reach = _expected_stats(tree, table, [0, N])
    with ub.Context(tree, table) as ctx:
        assert ctx.stat(ub.STAT_PAIR_BRANCH) == pb
        assert ctx.stat(ub.STAT_USEFUL) == us
        assert ctx.stat(ub.STAT_BRANCHES_KEPT) == kept
        assert ctx.stat(ub.STAT_MAX_REACH) == reach


# ------------------------------------------------------------------ streamed output

@pytest.mark.parametrize("n", [256, 255])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_streamed_output_equals_direct(small, n, precision):
    """unifrac_run_streamed (chunks of 7 stripes, and one chunk) gives the
    matrices of the FP64 oracle element by element within the precision's
    tolerance, and bit for bit those of unifrac_run, both layouts, every
    variant; odd and even N."""
    import torch
    w, ref_small = small
    table = synth.dense_to_table(w.table.dense()[:, :n], w.table.feature_node) \
        if n != w.table.n_samples else w.table
    ref = {v: (ref_small[v] if n == w.table.n_samples else oracle.unifrac_full(w.tree, table, v))
           for v in VARIANTS}
    iu = np.triu_indices(n, 1)
    with ub.Context(w.tree, table) as ctx:
        for layout in (ub.OUT_CONDENSED, ub.OUT_FULL):
            want = {v: (ref[v][iu] if layout == ub.OUT_CONDENSED else ref[v].reshape(-1))
                    for v in VARIANTS}
            want[ub.BOTH] = np.concatenate([want[ub.UNWEIGHTED], want[ub.WEIGHTED_NORMALIZED]])
            for variant in (ub.UNWEIGHTED, ub.WEIGHTED_NORMALIZED, ub.BOTH):
                direct = ctx.run(variant, precision, layout)
                torch.cuda.synchronize()
                direct = direct.cpu().numpy()
                for chunk in (7, 10_000):
                    got = ctx.run_streamed(variant, precision, layout, chunk)
                    assert got.shape == want[variant].shape
                    err = float(np.max(np.abs(got.astype(np.float64) - want[variant])))
                    assert err <= TOL[precision], f"max abs err {err:.3e}"
                    np.testing.assert_array_equal(got, direct)
        assert ctx.stat(ub.STAT_DEVICE_ERROR) == 0


@pytest.mark.parametrize("n", [256, 255])
def test_streamed_pinned_output_equals_pageable(small, n):
    """Into page-locked memory the full layout goes by 2D copies straight
    into the output (the rows whose runs wrap past column n through the host):
    the same bytes as into pageable memory, which the host places from row
    runs; both precisions, odd and even N, chunks of 1, 7 and all stripes
    (a ragged last chunk), and the condensed layout alongside."""
    import torch
    w, ref_small = small
    table = synth.dense_to_table(w.table.dense()[:, :n], w.table.feature_node) \
        if n != w.table.n_samples else w.table
    with ub.Context(w.tree, table) as ctx:
        for precision in PRECISIONS:
            dt = torch.float64 if precision == ub.FP64 else torch.float32
            for layout in (ub.OUT_FULL, ub.OUT_CONDENSED):
                nb = ctx.output_bytes(precision, layout) * 2
                for chunk in (1, 7, 10_000):
                    pageable = ctx.run_streamed(ub.BOTH, precision, layout, chunk)
                    pinned = torch.full((nb // dt.itemsize,), float("nan"), dtype=dt).pin_memory()
                    got = ctx.run_streamed(ub.BOTH, precision, layout, chunk, out=pinned.numpy())
                    np.testing.assert_array_equal(got, pageable)
        assert ctx.stat(ub.STAT_DEVICE_ERROR) == 0


def test_streamed_merge_threads_change_nothing(small):
    """UNIFRAC_OPT_HOST_THREADS sets the stripe merge's host threads (0: the
    CPUs the process may use): 1, 3 and 0 threads give the same bytes, full
    and condensed, odd N with a ragged last chunk; values outside 0 .. 256
    are rejected and leave the option as it was."""
    w, _ = small
    n = 255
    table = synth.dense_to_table(w.table.dense()[:, :n], w.table.feature_node)
    with ub.Context(w.tree, table) as ctx:
        assert ctx.get_option(ub.OPT_HOST_THREADS) == 0
        for bad in (-1, 257):
            with pytest.raises(ub.UniFracError):
                ctx.set_option(ub.OPT_HOST_THREADS, bad)
        assert ctx.get_option(ub.OPT_HOST_THREADS) == 0
        for layout in (ub.OUT_FULL, ub.OUT_CONDENSED):
            got = {}
            for threads in (1, 3, 0):
                ctx.set_option(ub.OPT_HOST_THREADS, threads)
                assert ctx.get_option(ub.OPT_HOST_THREADS) == threads
                got[threads] = ctx.run_streamed(ub.BOTH, ub.MIXED, layout, 9)
            np.testing.assert_array_equal(got[1], got[3])
            np.testing.assert_array_equal(got[1], got[0])
        assert ctx.stat(ub.STAT_DEVICE_ERROR) == 0


def test_streamed_output_rejects_bad_calls(small):
    import torch
    w, _ = small
    with ub.Context(w.tree, w.table) as ctx:
        with pytest.raises(ub.UniFracError):
            ctx.run_streamed(ub.UNWEIGHTED, ub.MIXED, ub.OUT_STRIPES, 4)
        with pytest.raises(ub.UniFracError):
            ctx.run_streamed(ub.UNWEIGHTED, ub.MIXED, ub.OUT_CONDENSED, 0)
        dev = torch.zeros(w.table.n_samples ** 2, dtype=torch.float32, device="cuda")
        with pytest.raises(ub.UniFracError):  # device memory
            ctx.run_streamed(ub.UNWEIGHTED, ub.MIXED, ub.OUT_FULL, 4, out=dev)
        small_out = np.zeros(10, np.float32)
        with pytest.raises(ub.UniFracError):
            ctx.run_streamed(ub.UNWEIGHTED, ub.MIXED, ub.OUT_FULL, 4, out=small_out)
    rng = np.random.default_rng(5)
    tree = synth.yule_tree(60, rng, 0.1)
    dense = (rng.random((60, 20)) < 0.3) * rng.integers(1, 9, (60, 20))
    table = synth.dense_to_table(dense, tree.tips())
    table.study_offsets = np.array([0, 9, 20], np.int32)
    with ub.Context(tree, table) as ctx:
        with pytest.raises(ub.UniFracError):  # several studies
            ctx.run_streamed(ub.UNWEIGHTED, ub.MIXED, ub.OUT_CONDENSED, 4)


# ------------------------------------------------------------------ PCoA

def test_pcoa_recovers_planar_configuration_on_gpu():
    """Distances of points in the plane: two eigenvalues (the squared
    singular values of the centred points), the rest ~0, and the first two
    coordinates reproduce the distances."""
    import torch
    from oracle import pcoa as opc
    rng = np.random.default_rng(8)
    X = rng.normal(size=(300, 2)) * np.array([2.0, 0.7])
    D = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    lam, C = ub.unifrac_pcoa(torch.from_numpy(D).cuda(), k=4, iters=8, seed=1)
    sv2 = np.linalg.svd(X - X.mean(axis=0), compute_uv=False) ** 2
    np.testing.assert_allclose(lam[:2], sv2, rtol=1e-5)
    assert np.all(np.abs(lam[2:]) <= 1e-5 * lam[0])
    Dc = np.sqrt(((C[:, None, :2] - C[None, :, :2]) ** 2).sum(-1))
    np.testing.assert_allclose(Dc, D, atol=1e-4 * D.max())
    lam_o, _ = opc.pcoa(D, 4)
    np.testing.assert_allclose(lam[:2], lam_o[:2], rtol=1e-5)


@pytest.mark.parametrize("variant", VARIANTS)
def test_pcoa_of_unifrac_matrix_matches_oracle(small, variant):
    """PCoA of the GPU UniFrac matrix (FP32, full layout) against the FP64
    oracle ordination of the same matrix: leading eigenvalues, and the
    coordinates of well-separated components up to sign."""
    import torch
    from oracle import pcoa as opc
    w, _ = small
    n = w.table.n_samples
    with ub.Context(w.tree, w.table) as ctx:
        D = ctx.run(variant, ub.MIXED, ub.OUT_FULL)
        torch.cuda.synchronize()
        k = 6
        lam, C = ub.unifrac_pcoa(D, k=k, iters=16, seed=7)
        lam2, C2 = ub.unifrac_pcoa(D, k=k, iters=16, seed=7)
    np.testing.assert_array_equal(lam, lam2)  # reproducible from the seed
    np.testing.assert_array_equal(C, C2)
    Dn = D.cpu().numpy().astype(np.float64).reshape(n, n)
    lam_o, C_o = opc.pcoa(Dn, k + 1)
    np.testing.assert_allclose(lam, lam_o[:k], rtol=2e-4, atol=1e-6 * lam_o[0])
    for c in range(k):
        gap = min(abs(lam_o[c] - lam_o[c + 1]), abs(lam_o[c] - lam_o[c - 1]) if c else np.inf)
        if gap < 0.05 * lam_o[c]:
            continue  # nearly degenerate: the axis itself is not determined
        sgn = np.sign(np.dot(C[:, c], C_o[:, c])) or 1.0
        np.testing.assert_allclose(sgn * C[:, c], C_o[:, c], atol=2e-3 * np.abs(C_o[:, c]).max())


def test_pcoa_rejects_bad_arguments():
    import torch
    D = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(ub.UniFracError):
        ub.unifrac_pcoa(D, k=5)  # k > n
    with pytest.raises(ub.UniFracError):
        ub.unifrac_pcoa(D, k=2, iters=-1)
    with pytest.raises(ValueError):
        ub.unifrac_pcoa(D.cpu(), k=2)


# ------------------------------------------------------------------ Mantel test

MANTEL_TOL = {ub.FP64: 1e-12, ub.MIXED: 2e-6}


def _mantel_perms(n, m, seed):
    rng = np.random.default_rng(seed)
    return np.array([rng.permutation(n) for _ in range(m)], dtype=np.int32).reshape(m, n)


def _point_matrices(n, seed, dtype):
    """Two correlated Euclidean distance matrices of random points (full n x n)."""
    import scipy.spatial.distance as ssd
    rng = np.random.default_rng(seed)
    a = rng.random((n, 3))
    b = a + 0.3 * rng.random((n, 3))
    return ssd.cdist(a, a).astype(dtype), ssd.cdist(b, b).astype(dtype)


def _check_mantel(got, want, tol):
    r, stats, p = got
    r_o, stats_o, p_o = want
    if np.isnan(r_o):
        assert np.isnan(r) and np.isnan(p) and np.isnan(stats).all()
        return
    assert abs(r - r_o) <= tol, (r, r_o)
    np.testing.assert_allclose(stats, stats_o, rtol=0, atol=tol)
    if np.isnan(p_o):
        assert np.isnan(p)
    elif not np.any(np.abs(np.abs(stats_o) - abs(r_o)) <= 2 * tol):
        assert p == p_o  # same decisions unless a statistic ties |r| within rounding


def _mantel_oracle(X, Y, perms, method):
    from oracle import mantel as om
    n = X.shape[0]
    iu = np.triu_indices(n, 1)
    return om.mantel(X.astype(np.float64)[iu], Y.astype(np.float64)[iu], n, perms, method)


@pytest.mark.parametrize("method", ["pearson", "spearman"])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_mantel_unifrac_matrices_match_oracle(small, method, precision):
    """Unweighted against weighted UniFrac of the same samples (the paper's
    use: do two distance matrices of one set of samples agree?), 99
    permutations, against the FP64 oracle on the same matrices."""
    import torch
    w, _ = small
    n = w.table.n_samples
    with ub.Context(w.tree, w.table) as ctx:
        X = ctx.run(ub.UNWEIGHTED, precision, ub.OUT_FULL)
        Y = ctx.run(ub.WEIGHTED_NORMALIZED, precision, ub.OUT_FULL)
    torch.cuda.synchronize()
    perms = _mantel_perms(n, 99, 21)
    got = ub.unifrac_mantel(X, Y, perms, method)
    again = ub.unifrac_mantel(X, Y, perms, method)
    assert got[0] == again[0] and got[2] == again[2]  # deterministic
    np.testing.assert_array_equal(got[1], again[1])
    Xn = X.cpu().numpy().reshape(n, n)
    Yn = Y.cpu().numpy().reshape(n, n)
    _check_mantel(got, _mantel_oracle(Xn, Yn, perms, method), MANTEL_TOL[precision])
    assert got[0] > 0.2  # the two UniFrac variants agree on these samples


def _row_bytes(n, precision):
    es = 8 if precision == ub.FP64 else 4
    return ((n + 16 // es + 3) & ~3) * es


@pytest.mark.parametrize("budget", [None, "0"])
@pytest.mark.parametrize("n", [3, 5, 37, 301])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_mantel_short_rows_and_ragged_sizes(n, budget, precision, monkeypatch):
    """Short rows (the small-block launch shape; with a zero staging budget,
    y read from global memory) at sizes whose rows start off the 16-byte
    grid, Pearson and Spearman."""
    import torch
    if budget is not None:
        monkeypatch.setenv("UNIFRAC_MANTEL_SMEM_BYTES", budget)
    dt = np.float64 if precision == ub.FP64 else np.float32
    X, Y = _point_matrices(n, 30 + n, dt)
    perms = _mantel_perms(n, 21, 31 + n)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    for method in ("pearson", "spearman"):
        got = ub.unifrac_mantel(Xd, Yd, perms, method)
        _check_mantel(got, _mantel_oracle(X, Y, perms, method), MANTEL_TOL[precision])


_LONG_ROW_ORACLE = {}


@pytest.mark.parametrize("shape", ["two_per_sm", "one_per_sm", "global"])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_mantel_long_row_launch_shapes(shape, precision, monkeypatch):
    """n = 6,501 (rows past the short-row limit; 1,024-thread blocks): two
    blocks per SM, one (budget between one and two rows), and no staging,
    against the oracle with 3 permutations (plus a 37-permutation run that
    spans several batches of the same launch)."""
    import torch
    n = 6501
    rb = _row_bytes(n, precision)
    if shape == "one_per_sm":
        monkeypatch.setenv("UNIFRAC_MANTEL_SMEM_BYTES", str(rb + 64))
    elif shape == "global":
        monkeypatch.setenv("UNIFRAC_MANTEL_SMEM_BYTES", "0")
    dt = np.float64 if precision == ub.FP64 else np.float32
    X, Y = _point_matrices(n, 80, dt)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    perms = _mantel_perms(n, 37, 81)
    r, stats, p = ub.unifrac_mantel(Xd, Yd, perms)
    if precision not in _LONG_ROW_ORACLE:
        _LONG_ROW_ORACLE[precision] = _mantel_oracle(X, Y, perms[:3], "pearson")
    r_o, stats_o, _ = _LONG_ROW_ORACLE[precision]
    _check_mantel((r, stats[:3], p), (r_o, stats_o, p), MANTEL_TOL[precision])
    r3, stats3, _ = ub.unifrac_mantel(Xd, Yd, perms[:3])
    assert r3 == r  # the identity's sum does not depend on the batch
    np.testing.assert_array_equal(stats3, stats[:3])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_mantel_spearman_heavy_ties(precision):
    """Distances rounded to one decimal: long runs of equal values, whose
    members share the mean rank."""
    import torch
    dt = np.float64 if precision == ub.FP64 else np.float32
    X, Y = _point_matrices(400, 41, np.float64)
    X, Y = np.round(X, 1).astype(dt), np.round(Y, 1).astype(dt)
    perms = _mantel_perms(400, 15, 42)
    got = ub.unifrac_mantel(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), perms,
                            "spearman")
    _check_mantel(got, _mantel_oracle(X, Y, perms, "spearman"), MANTEL_TOL[precision])


def test_mantel_degenerate_cases():
    """Constant matrix (no correlation: NaN), no permutations (p NaN), y = x
    with identity relabellings (r = 1, p = 1), all six relabellings of n = 3."""
    import itertools
    import torch
    X, _ = _point_matrices(24, 50, np.float64)
    Xd = torch.from_numpy(X).cuda()
    C = torch.full((24, 24), 0.5, dtype=torch.float64, device="cuda")
    perms = _mantel_perms(24, 5, 51)
    _check_mantel(ub.unifrac_mantel(Xd, C, perms), _mantel_oracle(X, C.cpu().numpy(), perms,
                                                                   "pearson"), 1e-12)
    r, stats, p = ub.unifrac_mantel(Xd, Xd, perms[:0])
    assert abs(r - 1.0) <= 1e-12 and np.isnan(p) and stats.shape == (0,)
    ident = np.tile(np.arange(24, dtype=np.int32), (4, 1))
    r, stats, p = ub.unifrac_mantel(Xd, Xd, ident)
    assert p == 1.0 and np.allclose(stats, 1.0, atol=1e-12)
    X3, Y3 = _point_matrices(3, 52, np.float64)
    all3 = np.array(list(itertools.permutations(range(3))), dtype=np.int32)
    for method in ("pearson", "spearman"):
        got = ub.unifrac_mantel(torch.from_numpy(X3).cuda(), torch.from_numpy(Y3).cuda(), all3,
                                method)
        _check_mantel(got, _mantel_oracle(X3, Y3, all3, method), 1e-12)


def test_mantel_rejects_bad_arguments():
    import torch
    X, Y = _point_matrices(10, 60, np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    good = _mantel_perms(10, 3, 61)
    bad = good.copy()
    bad[1, 0] = bad[1, 1]  # not a permutation
    with pytest.raises(ub.UniFracError):
        ub.unifrac_mantel(Xd, Yd, bad)
    out_of_range = good.copy()
    out_of_range[2, 4] = 10
    with pytest.raises(ub.UniFracError):
        ub.unifrac_mantel(Xd, Yd, out_of_range)
    two = torch.zeros((2, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(ub.UniFracError):
        ub.unifrac_mantel(two, two, np.zeros((1, 2), np.int32))  # n < 3
    with pytest.raises(ValueError):
        ub.unifrac_mantel(Xd, Yd.double(), good)  # mixed dtypes
    with pytest.raises(ValueError):
        ub.unifrac_mantel(Xd.cpu(), Yd.cpu(), good)  # host tensors
    with pytest.raises(ValueError):
        ub.unifrac_mantel(Xd, Yd, good, method="kendall")


def test_mantel_large_matrices_sampled_permutations():
    """n = 12,000 (72 M pairs, rows of y staged in two 48 KB buffers): the
    statistic and two permuted statistics against the oracle."""
    import torch
    n = 12000
    X, Y = _point_matrices(n, 70, np.float32)
    perms = _mantel_perms(n, 2, 71)
    got = ub.unifrac_mantel(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), perms)
    _check_mantel(got, _mantel_oracle(X, Y, perms, "pearson"), MANTEL_TOL[ub.MIXED])


# ------------------------------------------------------------------ bounded device waits

def test_bounded_wait_runs_out_and_device_stays_usable(small):
    """The bounded mbarrier wait of the tensor-core kernel, run on a barrier
    that nothing completes with a 20 ms limit, gives up and records
    UNIFRAC_E_DEVICE_TIMEOUT; the device then computes as before."""
    import time
    t0 = time.perf_counter()
    status = ub.unifrac_check_bounded_wait(20000)
    elapsed = time.perf_counter() - t0
    assert status == -8  # UNIFRAC_E_DEVICE_TIMEOUT
    assert 0.02 <= elapsed < 5.0
    w, ref = small
    N = w.table.n_samples
    got = run(w.tree, w.table, ub.UNWEIGHTED, ub.MIXED).reshape(N, N)
    check_full(got, ref[ub.UNWEIGHTED], ub.MIXED)


def test_mantel_batches_beyond_one_launch():
    """1,048,600 permutations of 3 samples: 65,538 batches of 16, more than
    one launch's 65,535 grid rows, so the cross sums run as two launches.
    Each of the six distinct relabellings is evaluated by the oracle once."""
    import itertools
    import torch
    from oracle import mantel as om
    X, Y = _point_matrices(3, 90, np.float64)
    iu = np.triu_indices(3, 1)
    distinct = np.array(list(itertools.permutations(range(3))), dtype=np.int32)
    pick = np.random.default_rng(91).integers(0, 6, size=1_048_600)
    perms = distinct[pick]
    r, stats, p = ub.unifrac_mantel(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), perms)
    r_o, stats6, _ = om.mantel(X[iu], Y[iu], 3, distinct)
    assert abs(r - r_o) <= 1e-12
    np.testing.assert_allclose(stats, stats6[pick], rtol=0, atol=1e-12)
    hits = np.count_nonzero(np.abs(stats6[pick]) >= abs(r_o))
    assert p == (1.0 + hits) / (len(perms) + 1.0)


def test_pcoa_all_components():
    """k = n (the subspace is the whole space): every eigenvalue of the
    double-centred matrix, against the oracle."""
    import torch
    from oracle import pcoa as opc
    X, _ = _point_matrices(12, 92, np.float64)
    lam, C = ub.unifrac_pcoa(torch.from_numpy(X).cuda(), k=12, iters=4, seed=3)
    lam_o, _ = opc.pcoa(X, 12)
    np.testing.assert_allclose(lam, lam_o, rtol=1e-5, atol=1e-6 * abs(lam_o[0]))


# ------------------------------------------------------------------ table forms at create

def _with_explicit_zeros(table, seed):
    """The same table with explicit zero counts inserted in about half of the
    rows (at sample ids the row does not use), rows kept sorted."""
    rng = np.random.default_rng(seed)
    ip, ix, ct = [0], [], []
    for f in range(table.n_features):
        lo, hi = int(table.indptr[f]), int(table.indptr[f + 1])
        idx, cnt = list(table.indices[lo:hi]), list(table.counts[lo:hi])
        if rng.random() < 0.5:
            free = np.setdiff1d(np.arange(table.n_samples), idx)
            for s in rng.choice(free, size=min(3, len(free)), replace=False):
                idx.append(int(s))
                cnt.append(0)
        order = np.argsort(idx, kind="stable")
        ix += [idx[k] for k in order]
        ct += [cnt[k] for k in order]
        ip.append(len(ix))
    return synth.Table(table.n_features, table.n_samples, np.array(ip, np.int64),
                       np.array(ix, np.int32), np.array(ct, np.int32), table.feature_node,
                       table.study_offsets)


def _with_shuffled_rows(table, seed):
    """The same table with every row's entries in a random order."""
    rng = np.random.default_rng(seed)
    ix, ct = table.indices.copy(), table.counts.copy()
    for f in range(table.n_features):
        lo, hi = int(table.indptr[f]), int(table.indptr[f + 1])
        p = rng.permutation(hi - lo) + lo
        ix[lo:hi], ct[lo:hi] = table.indices[p], table.counts[p]
    return synth.Table(table.n_features, table.n_samples, table.indptr.copy(), ix, ct,
                       table.feature_node, table.study_offsets)


@pytest.mark.parametrize("studies", [1, 3])
@pytest.mark.parametrize("form", ["zeros", "shuffled"])
def test_table_forms_give_the_same_matrices(small, form, studies):
    """Explicit zero counts (copied without them) and unsorted rows (the
    sequential pass) give exactly the matrices of the canonical table (whose
    entries are uploaded as they are), with one study and with three."""
    w, _ = small
    table = w.table
    if studies > 1:
        n = table.n_samples
        table = synth.Table(table.n_features, n, table.indptr, table.indices, table.counts,
                            table.feature_node, np.array([0, n // 3, 2 * n // 3, n], np.int32))
    other = _with_explicit_zeros(table, 95) if form == "zeros" else _with_shuffled_rows(table, 96)
    for variant in VARIANTS:
        a = run(w.tree, table, variant, ub.MIXED, layout=ub.OUT_CONDENSED)
        b = run(w.tree, other, variant, ub.MIXED, layout=ub.OUT_CONDENSED)
        np.testing.assert_array_equal(a, b)
