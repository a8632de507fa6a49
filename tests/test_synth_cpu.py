"""The seeded input generator against the workload recipe it states (no GPU).

Every parity test and the bench draw their inputs from
paper_2107_05397_b300/synth.py.  These checks hold the generated workloads to
the recipe: tree sizes, a valid postorder with the root last, branch lengths
with the stated exponential mean, the stated fraction of non-zero cells,
counts of at least 1 that fit int32, at least one feature per sample, one
feature per tip, Zipf-skewed feature popularity where the recipe says so,
study sizes within the stated log-uniform range, and the same arrays on every
draw (seeded).
"""
import numpy as np
import pytest

from paper_2107_05397_b300 import synth


def _valid_postorder(tree):
    n = tree.n_nodes
    assert tree.parent[n - 1] == -1
    k = np.arange(n - 1)
    assert np.all(tree.parent[:-1] > k) and np.all(tree.parent[:-1] < n)
    assert np.all(np.isfinite(tree.length)) and np.all(tree.length[:-1] >= 0)


def _occurrences(table):
    return np.bincount(np.repeat(np.arange(table.n_features), np.diff(table.indptr)),
                       minlength=table.n_features)


def _check_table(table, tree):
    assert table.indptr[0] == 0 and table.indptr[-1] == table.nnz
    assert np.all(np.diff(table.indptr) >= 0)
    assert np.all((table.indices >= 0) & (table.indices < table.n_samples))
    assert np.all(table.counts >= 1) and np.all(table.counts <= 2**31 - 1)
    # one feature per tip, every feature on a tip
    fn = table.feature_node
    assert np.unique(fn).shape[0] == fn.shape[0]
    assert np.all(np.isin(fn, tree.tips()))
    # no duplicate (feature, sample) cell: sample ids strictly increase per row
    for f in range(0, table.n_features, max(1, table.n_features // 64)):
        seg = table.indices[table.indptr[f]:table.indptr[f + 1]]
        assert np.all(np.diff(seg) > 0)
    # every sample holds at least one feature
    assert np.all(np.bincount(table.indices, minlength=table.n_samples) >= 1)


@pytest.mark.parametrize("name,tips,mean_len,samples,density,zipf", [
    ("tips1024_samples256", 1024, 0.1, 256, 0.03, False),
    ("tips32768_samples4096", 32768, 0.1, 4096, 0.01, True),
])
def test_named_workload_follows_its_recipe(name, tips, mean_len, samples, density, zipf):
    w = synth.make_workload(name)
    tree, table = w.tree, w.table
    assert tree.tips().shape[0] == tips and tree.n_nodes == 2 * tips - 1  # binary tree
    _valid_postorder(tree)
    # Exp(mean) lengths: the sample mean within 5 standard errors
    L = tree.length[:-1]
    assert abs(L.mean() - mean_len) < 5 * mean_len / np.sqrt(L.shape[0])
    assert table.n_features == tips and table.n_samples == samples
    _check_table(table, tree)
    # Binomial(F, density) features per sample (at least 1): the fill within 5 %
    fill = table.nnz / (table.n_features * table.n_samples)
    assert abs(fill - density) < 0.05 * density
    occ = _occurrences(table)
    if zipf:
        # Zipf popularity: the most popular features sit in almost every
        # sample, the typical feature in few
        assert occ.max() >= 0.9 * samples
        assert np.median(occ) < 0.1 * samples
    else:
        # uniform popularity: occurrences stay near samples x density
        assert occ.max() < 4 * samples * density


def test_workloads_are_seeded():
    a = synth._make_workload("tips1024_samples256")
    b = synth._make_workload("tips1024_samples256")
    for x, y in ((a.tree.parent, b.tree.parent), (a.tree.length, b.tree.length),
                 (a.table.indptr, b.table.indptr), (a.table.indices, b.table.indices),
                 (a.table.counts, b.table.counts), (a.table.feature_node, b.table.feature_node)):
        np.testing.assert_array_equal(x, y)


def test_truncated_workload_is_a_prefix_of_the_samples():
    """n_samples truncation keeps the first samples of the full draw (tests
    that run a smaller case of a workload compare the same columns)."""
    full = synth._make_workload("tips1024_samples256")
    part = synth._make_workload("tips1024_samples256", n_samples=100)
    np.testing.assert_array_equal(part.tree.parent, full.tree.parent)
    np.testing.assert_array_equal(part.table.feature_node, full.table.feature_node)
    np.testing.assert_array_equal(part.table.dense(), full.table.dense()[:, :100])


def test_batched_studies_follow_their_recipe():
    """Studies of log-uniform size in [200, 6000] sharing one 50,000-tip tree,
    each at its own density in [0.5 %, 3 %] (six studies drawn here; the
    workload has 64)."""
    w = synth.make_batched("tips50000_studies64", n_studies=6)
    tree, table = w.tree, w.table
    assert tree.tips().shape[0] == 50000
    _valid_postorder(tree)
    _check_table(table, tree)
    so = table.study_offsets
    assert so is not None and so[0] == 0 and so[-1] == table.n_samples and len(so) == 7
    sizes = np.diff(so)
    assert np.all((sizes >= 200) & (sizes <= 6000))
    per_sample = np.bincount(table.indices, minlength=table.n_samples)
    for s in range(6):
        fill = per_sample[so[s]:so[s + 1]].mean() / table.n_features
        assert 0.005 * 0.9 < fill < 0.03 * 1.1
