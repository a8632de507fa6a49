"""Pins for the FP64 oracle against facts that do not come from the oracle.

Each test checks the oracle against something fixed by the paper's problem
statement (Section II) or by mathematics: a hand-derived worked example,
brute-force ancestor walks, star-tree closed forms that reduce to textbook
distances computed by scipy (Jaccard, Bray-Curtis), the earth mover's
distance of the weighted numerator (a transport linear program), Faith's
phylogenetic diversity, the tip-depth identity of the weighted denominator, and metric
invariants.  A dropped term, wrong sign, wrong index or swapped operand in the
oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.spatial.distance as ssd

import oracle
from paper_2107_05397_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
UW, WN = oracle.UNWEIGHTED, oracle.WEIGHTED_NORMALIZED


def _children(parent):
    kids = [[] for _ in range(parent.shape[0])]
    for v, p in enumerate(parent):
        if p >= 0:
            kids[p].append(v)
    return kids


def brute_embedding(tree, table):
    """w[node, sample], p[node, sample] by walking up from every tip."""
    n = tree.n_nodes
    dense = table.dense()
    N = table.n_samples
    tot = dense.sum(axis=0).astype(np.float64)
    w = np.zeros((n, N))
    cnt = np.zeros((n, N))
    for f in range(table.n_features):
        v = int(table.feature_node[f])
        while v >= 0:  # every ancestor, including the tip itself
            cnt[v] += dense[f]
            v = int(tree.parent[v])
    with np.errstate(invalid="ignore", divide="ignore"):
        w = np.where(tot > 0, cnt / np.where(tot > 0, tot, 1), 0.0)
    return w, (cnt > 0).astype(np.uint8)


def branch_sets(tree, table):
    """Set of non-root branches on the root paths of each sample's tips."""
    dense = table.dense()
    root = tree.n_nodes - 1
    sets = []
    for i in range(table.n_samples):
        s = set()
        for f in np.nonzero(dense[:, i])[0]:
            v = int(table.feature_node[f])
            while v != root:
                s.add(v)
                v = int(tree.parent[v])
        sets.append(s)
    return sets


def depth(tree):
    """Root-to-node path length, root branch excluded."""
    d = np.zeros(tree.n_nodes)
    for v in range(tree.n_nodes - 2, -1, -1):  # parents before children
        d[v] = d[tree.parent[v]] + tree.length[v]
    return d


def cases():
    out = []
    for seed in range(6):
        rng = np.random.default_rng(1000 + seed)
        general = seed % 2 == 1
        tree, table = synth.random_case(rng, n_tips=4 + 2 * seed, n_samples=7,
                                        density=0.35, general=general,
                                        empty_samples=1 if seed == 2 else 0)
        out.append((tree, table))
    return out


# ---------------------------------------------------------------- worked example

def test_worked_example_golden():
    g = json.load(open(os.path.join(GOLDEN, "worked_example_7node.json")))
    tree = synth.Tree(parent=np.array(g["parent"], np.int32), length=np.array(g["length"]))
    table = synth.dense_to_table(np.array(g["dense_counts_features_by_samples"]),
                                 np.array(g["feature_node"], np.int32))
    np.testing.assert_allclose(oracle.unifrac_full(tree, table, UW), g["unweighted"],
                               rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.unifrac_full(tree, table, WN), g["weighted_normalized"],
                               rtol=0, atol=1e-15)


# ---------------------------------------------------------------- embedding

@pytest.mark.parametrize("k", range(6))
def test_embedding_matches_ancestor_walk(k):
    tree, table = cases()[k]
    w_ref, p_ref = brute_embedding(tree, table)
    for i in range(table.n_samples):
        w, p = oracle.embedding(tree, table, i)
        np.testing.assert_allclose(w, w_ref[:, i], rtol=0, atol=1e-15)
        np.testing.assert_array_equal(p, p_ref[:, i])


def test_embedding_postorder_range_identity():
    """In postorder numbering a subtree is the node range [b-size_b+1, b]."""
    rng = np.random.default_rng(7)
    tree, table = synth.random_case(rng, n_tips=12, n_samples=5, general=True)
    n = tree.n_nodes
    size = np.ones(n, dtype=np.int64)
    for v in range(n - 1):
        size[tree.parent[v]] += size[v]
    dense = table.dense()
    tip_count = np.zeros((n, table.n_samples))
    tip_count[table.feature_node] = dense
    prefix = np.vstack([np.zeros((1, table.n_samples)), np.cumsum(tip_count, axis=0)])
    tot = dense.sum(axis=0)
    for i in range(table.n_samples):
        w, _ = oracle.embedding(tree, table, i)
        below = prefix[np.arange(n) + 1, i] - prefix[np.arange(n) + 1 - size, i]
        np.testing.assert_allclose(w, below / tot[i] if tot[i] else 0 * below,
                                   rtol=0, atol=1e-15)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("equal", [True, False])
def test_star_tree_unweighted_is_jaccard(equal):
    rng = np.random.default_rng(11)
    F, N = 15, 9
    tree = synth.star_tree(F, 0.7)
    if not equal:
        tree.length[:-1] = rng.exponential(0.5, size=F)
    dense = (rng.random((F, N)) < 0.4) * rng.integers(1, 9, size=(F, N))
    table = synth.dense_to_table(dense, np.arange(F, dtype=np.int32))
    d = oracle.unifrac_full(tree, table, UW)
    for i in range(N):
        for j in range(N):
            a, b = dense[:, i] > 0, dense[:, j] > 0
            if not (a | b).any():
                ref = 0.0
            else:
                ref = ssd.jaccard(a, b, w=tree.length[:-1])
            assert abs(d[i, j] - ref) < 1e-14, (i, j, d[i, j], ref)


@pytest.mark.parametrize("equal", [True, False])
def test_star_tree_weighted_is_bray_curtis(equal):
    rng = np.random.default_rng(12)
    F, N = 13, 8
    tree = synth.star_tree(F, 0.3)
    if not equal:
        tree.length[:-1] = rng.exponential(0.5, size=F)
    dense = (rng.random((F, N)) < 0.5) * rng.integers(1, 50, size=(F, N))
    dense[:, 0] = 0
    dense[3, 0] = 4  # at least one non-empty
    table = synth.dense_to_table(dense, np.arange(F, dtype=np.int32))
    d = oracle.unifrac_full(tree, table, WN)
    for i in range(N):
        for j in range(N):
            u, v = dense[:, i].astype(float), dense[:, j].astype(float)
            if u.sum() == 0 and v.sum() == 0:
                ref = 0.0
            else:
                u = u / u.sum() if u.sum() else u
                v = v / v.sum() if v.sum() else v
                ref = ssd.braycurtis(u, v, w=tree.length[:-1])
            assert abs(d[i, j] - ref) < 1e-14, (i, j, d[i, j], ref)


@pytest.mark.parametrize("k", range(6))
def test_unweighted_from_branch_sets(k):
    """Unweighted = length of symmetric difference / length of union of the
    two samples' branch sets; Faith's PD is the length of one set."""
    tree, table = cases()[k]
    sets = branch_sets(tree, table)
    L = tree.length
    d = oracle.unifrac_full(tree, table, UW)
    for i in range(table.n_samples):
        for j in range(table.n_samples):
            sym = sum(L[b] for b in sets[i] ^ sets[j])
            uni = sum(L[b] for b in sets[i] | sets[j])
            ref = sym / uni if uni > 0 else 0.0
            assert abs(d[i, j] - ref) < 1e-13


@pytest.mark.parametrize("k", range(6))
def test_weighted_denominator_tip_depth_identity(k):
    """sum_b len_b w_bi = sum_f (c_fi / C_i) depth(tip_f); with a sample that
    has nothing in common, the weighted distance is 1 and its denominator is
    the sum of both mean tip depths."""
    tree, table = cases()[k]
    dep = depth(tree)
    dense = table.dense().astype(float)
    for i in range(table.n_samples):
        w, _ = oracle.embedding(tree, table, i)
        lhs = float(np.dot(tree.length[:-1], w[:-1]))
        tot = dense[:, i].sum()
        rhs = float(np.dot(dense[:, i] / tot, dep[table.feature_node])) if tot else 0.0
        assert abs(lhs - rhs) < 1e-13


def tip_path_lengths(tree, tips):
    """Tree path length between every two tips: depth(a) + depth(b) minus
    twice the depth of their deepest common ancestor (from ancestor sets)."""
    dep = depth(tree)
    anc = []
    for t in tips:
        s, v = set(), int(t)
        while v >= 0:
            s.add(v)
            v = int(tree.parent[v])
        anc.append(s)
    n = len(tips)
    C = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            lca_depth = max(dep[v] for v in anc[a] & anc[b])
            C[a, b] = dep[tips[a]] + dep[tips[b]] - 2.0 * lca_depth
    return C


@pytest.mark.parametrize("k", range(6))
def test_weighted_numerator_is_earth_movers_distance(k):
    """Weighted UniFrac's numerator sum_b len_b |w_bi - w_bj| is the earth
    mover's (Kantorovich) distance between the two samples' relative
    abundances on the tips, with the tree's path lengths as ground distance.
    The transport problem is solved as a linear program (scipy's HiGHS), and
    the denominator is the sum of the two mean tip depths, so
    d_ij * (D_i + D_j) must equal the transport cost."""
    from scipy.optimize import linprog
    tree, table = cases()[k]
    d = oracle.unifrac_full(tree, table, WN)
    dense = table.dense().astype(float)
    tips = table.feature_node.astype(np.int64)
    C = tip_path_lengths(tree, tips)
    dep = depth(tree)[tips]
    F = len(tips)
    # equality constraints of a transport plan T[f, g] >= 0 (row-major):
    # rows sum to p, columns sum to q
    A = np.zeros((2 * F, F * F))
    for f in range(F):
        A[f, f * F:(f + 1) * F] = 1.0
        A[F + f, f::F] = 1.0
    checked = 0
    for i in range(table.n_samples):
        for j in range(i + 1, table.n_samples):
            ti, tj = dense[:, i].sum(), dense[:, j].sum()
            if ti == 0 or tj == 0:
                continue
            p, q = dense[:, i] / ti, dense[:, j] / tj
            res = linprog(C.ravel(), A_eq=A, b_eq=np.concatenate([p, q]), bounds=(0, None),
                          method="highs")
            assert res.status == 0
            numer = d[i, j] * (float(p @ dep) + float(q @ dep))
            assert abs(numer - res.fun) < 1e-8, (i, j, numer, res.fun)
            checked += 1
    assert checked >= 10


def test_faith_pd_golden():
    g = json.load(open(os.path.join(GOLDEN, "worked_example_7node.json")))
    tree = synth.Tree(parent=np.array(g["parent"], np.int32), length=np.array(g["length"]))
    table = synth.dense_to_table(np.array(g["dense_counts_features_by_samples"]),
                                 np.array(g["feature_node"], np.int32))
    for i, (pd, td) in enumerate(zip(g["faith_pd"], g["tip_depth_mean"])):
        w, p = oracle.embedding(tree, table, i)
        assert abs(np.dot(tree.length[:-1], p[:-1]) - pd) < 1e-15
        assert abs(np.dot(tree.length[:-1], w[:-1]) - td) < 1e-15


def test_root_disjoint_samples_unweighted_one():
    """Features under different children of the root share no branch."""
    rng = np.random.default_rng(5)
    tree = synth.yule_tree(16, rng, 0.2)
    root = tree.n_nodes - 1
    kids = _children(tree.parent)[root]
    assert len(kids) == 2
    size = np.ones(tree.n_nodes, dtype=np.int64)
    for v in range(tree.n_nodes - 1):
        size[tree.parent[v]] += size[v]
    left = set(range(kids[0] - size[kids[0]] + 1, kids[0] + 1))
    tips = tree.tips()
    lt = [t for t in tips if t in left]
    rt = [t for t in tips if t not in left]
    fnode = np.array(lt + rt, dtype=np.int32)
    dense = np.zeros((len(fnode), 2), dtype=np.int64)
    dense[: len(lt), 0] = rng.integers(1, 5, size=len(lt))
    dense[len(lt):, 1] = rng.integers(1, 5, size=len(rt))
    table = synth.dense_to_table(dense, fnode)
    assert abs(oracle.unifrac_full(tree, table, UW)[0, 1] - 1.0) < 1e-15
    assert abs(oracle.unifrac_full(tree, table, WN)[0, 1] - 1.0) < 1e-15


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("variant", [UW, WN])
@pytest.mark.parametrize("k", range(6))
def test_metric_properties(variant, k):
    tree, table = cases()[k]
    d = oracle.unifrac_full(tree, table, variant)
    assert np.all(np.diag(d) == 0)
    np.testing.assert_array_equal(d, d.T)
    assert d.min() >= 0 and d.max() <= 1 + 1e-15
    if variant == UW:  # weighted Jaccard on branch sets is a metric
        N = d.shape[0]
        for a in range(N):
            for b in range(N):
                assert np.all(d[a, b] <= d[a, :] + d[:, b] + 1e-12)


@pytest.mark.parametrize("variant", [UW, WN])
def test_permuting_samples_permutes_matrix(variant):
    rng = np.random.default_rng(21)
    tree, table = synth.random_case(rng, n_tips=10, n_samples=9)
    dense = table.dense()
    perm = rng.permutation(table.n_samples)
    t2 = synth.dense_to_table(dense[:, perm], table.feature_node)
    d1 = oracle.unifrac_full(tree, table, variant)
    d2 = oracle.unifrac_full(tree, t2, variant)
    np.testing.assert_allclose(d2, d1[np.ix_(perm, perm)], rtol=0, atol=1e-15)


@pytest.mark.parametrize("variant", [UW, WN])
def test_feature_relabel_and_count_scaling(variant):
    rng = np.random.default_rng(22)
    tree, table = synth.random_case(rng, n_tips=10, n_samples=6)
    dense = table.dense()
    fperm = rng.permutation(table.n_features)
    t2 = synth.dense_to_table(dense[fperm], table.feature_node[fperm])
    scale = rng.integers(1, 7, size=table.n_samples)
    t3 = synth.dense_to_table(dense * scale[None, :], table.feature_node)
    d1 = oracle.unifrac_full(tree, table, variant)
    np.testing.assert_allclose(oracle.unifrac_full(tree, t2, variant), d1, rtol=0, atol=1e-15)
    np.testing.assert_allclose(oracle.unifrac_full(tree, t3, variant), d1, rtol=0, atol=1e-14)


@pytest.mark.parametrize("variant", [UW, WN])
def test_unary_split_and_zero_length_branch_change_nothing(variant):
    """Splitting a branch into two pieces of the same total length, or adding a
    zero-length pendant tip with no feature, leaves every distance unchanged."""
    rng = np.random.default_rng(23)
    tree, table = synth.random_case(rng, n_tips=8, n_samples=6)
    d1 = oracle.unifrac_full(tree, table, variant)
    n = tree.n_nodes
    v = int(rng.integers(0, n - 1))
    # build explicitly in postorder: insert u right after v (subtree of v stays contiguous)
    new_parent = np.empty(n + 1, np.int32)
    new_len = np.empty(n + 1)
    remap = np.arange(n) + (np.arange(n) > v)  # old id -> new id
    for k in range(n):
        p = int(tree.parent[k])
        new_parent[remap[k]] = -1 if p < 0 else remap[p]
        new_len[remap[k]] = tree.length[k]
    u = v + 1
    new_parent[u] = remap[tree.parent[v]]
    new_parent[v] = u
    new_len[u] = tree.length[v] * 0.3
    new_len[v] = tree.length[v] * 0.7
    t2 = synth.Tree(parent=new_parent, length=new_len)
    table2 = synth.coo_to_table(table.n_features, table.n_samples,
                                *np.nonzero(table.dense()),
                                table.dense()[np.nonzero(table.dense())],
                                remap[table.feature_node].astype(np.int32))
    np.testing.assert_allclose(oracle.unifrac_full(t2, table2, variant), d1, rtol=0, atol=1e-13)
    # zero-length pendant tip without a feature: appended as node 0
    p3 = np.concatenate([[tree.parent[0] + 1], tree.parent + 1]).astype(np.int32)
    p3[-1] = -1
    l3 = np.concatenate([[0.0], tree.length])
    t3 = synth.Tree(parent=p3, length=l3)
    table3 = synth.Table(table.n_features, table.n_samples, table.indptr, table.indices,
                         table.counts, (table.feature_node + 1).astype(np.int32))
    np.testing.assert_allclose(oracle.unifrac_full(t3, table3, variant), d1, rtol=0, atol=1e-15)


def test_empty_samples():
    rng = np.random.default_rng(24)
    tree, table = synth.random_case(rng, n_tips=9, n_samples=5, empty_samples=2)
    dense = table.dense()
    empty = np.nonzero(dense.sum(axis=0) == 0)[0]
    full = np.nonzero(dense.sum(axis=0) > 0)[0]
    assert len(empty) == 2 and len(full) > 0
    for variant in (UW, WN):
        d = oracle.unifrac_full(tree, table, variant)
        assert d[empty[0], empty[1]] == 0.0
        for j in full:
            assert d[empty[0], j] == 1.0


def test_rows_equal_pairs_and_thread_count():
    rng = np.random.default_rng(25)
    tree, table = synth.random_case(rng, n_tips=20, n_samples=12)
    rows = [3, 0, 11]
    out, used = oracle.unifrac_rows(tree, table, WN, rows, n_threads=2)
    assert used >= 1
    pi = np.repeat(rows, table.n_samples)
    pj = np.tile(np.arange(table.n_samples), len(rows))
    np.testing.assert_array_equal(oracle.unifrac_pairs(tree, table, WN, pi, pj),
                                  out.reshape(-1))


def test_invalid_inputs_rejected():
    tree = synth.Tree(parent=np.array([2, 2, -1], np.int32), length=np.ones(3))
    table = synth.dense_to_table(np.array([[1], [2]]), np.array([0, 1], np.int32))
    bad_tree = synth.Tree(parent=np.array([2, 0, -1], np.int32), length=np.ones(3))
    with pytest.raises(ValueError):
        oracle.unifrac_full(bad_tree, table, UW)
    internal = synth.dense_to_table(np.array([[1], [2]]), np.array([0, 2], np.int32))
    with pytest.raises(ValueError):
        oracle.unifrac_full(tree, internal, UW)


def test_duplicate_cells_and_shared_tips_rejected():
    """A table with one (feature, sample) cell listed twice, or with two
    features on one tip, is malformed and rejected; it is not read as the sum
    of the entries (the readings of the problem statement for duplicates and
    for a tip as one taxon)."""
    tree = synth.Tree(parent=np.array([2, 2, -1], np.int32), length=np.ones(3))
    fnode = np.array([0, 1], np.int32)
    ok = synth.Table(n_features=2, n_samples=2, indptr=np.array([0, 2, 3], np.int64),
                     indices=np.array([0, 1, 1], np.int32),
                     counts=np.array([3, 1, 2], np.int32), feature_node=fnode)
    d = oracle.unifrac_full(tree, ok, WN)
    # sample 0: feature 0 only (w = 1, 0 on tips 0, 1); sample 1: features 0
    # and 1 with counts 1 and 2 (w = 1/3, 2/3): (2/3 + 2/3) / (4/3 + 2/3)
    assert d[0, 1] == pytest.approx(2.0 / 3.0, abs=1e-15)
    for variant in (UW, WN):
        dup = synth.Table(n_features=2, n_samples=2, indptr=np.array([0, 3, 4], np.int64),
                          indices=np.array([0, 1, 1, 1], np.int32),
                          counts=np.array([3, 1, 1, 2], np.int32), feature_node=fnode)
        with pytest.raises(ValueError):
            oracle.unifrac_full(tree, dup, variant)
        shared = synth.Table(n_features=2, n_samples=2, indptr=np.array([0, 1, 2], np.int64),
                             indices=np.array([0, 1], np.int32),
                             counts=np.array([3, 1], np.int32),
                             feature_node=np.array([0, 0], np.int32))
        with pytest.raises(ValueError):
            oracle.unifrac_full(tree, shared, variant)


@pytest.mark.parametrize("variant", [UW, WN])
def test_root_branch_length_is_ignored(variant):
    """Reading of the paper's silence on the root: its length never counts."""
    rng = np.random.default_rng(26)
    tree, table = synth.random_case(rng, n_tips=9, n_samples=6)
    d1 = oracle.unifrac_full(tree, table, variant)
    t2 = synth.Tree(parent=tree.parent, length=tree.length.copy())
    t2.length[-1] = 5.0
    np.testing.assert_array_equal(oracle.unifrac_full(t2, table, variant), d1)


# ------------------------------------------------------------------ PCoA oracle

def test_pcoa_recovers_planar_configuration():
    """Classical MDS recovers points in the plane up to a rigid motion: the
    coordinates reproduce the distances, the two non-zero eigenvalues are the
    squared singular values of the centred points, the rest vanish."""
    from oracle import pcoa
    rng = np.random.default_rng(3)
    X = rng.normal(size=(40, 2)) * np.array([3.0, 1.0])
    D = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    lam, C = pcoa.pcoa(D, 5)
    Dc = np.sqrt(((C[:, None, :2] - C[None, :, :2]) ** 2).sum(-1))
    np.testing.assert_allclose(Dc, D, atol=1e-10)
    Xc = X - X.mean(axis=0)
    sv = np.linalg.svd(Xc, compute_uv=False)
    np.testing.assert_allclose(lam[:2], sv ** 2, rtol=1e-10)
    assert np.all(np.abs(lam[2:]) < 1e-9)


def test_pcoa_eigenvalues_sum_to_trace():
    """sum of all eigenvalues = trace(B) = (1/n) sum_{i<j} d_ij^2."""
    from oracle import pcoa
    rng = np.random.default_rng(4)
    n = 25
    M = rng.random((n, n))
    D = M + M.T
    np.fill_diagonal(D, 0.0)
    lam, _ = pcoa.pcoa(D, n)
    iu = np.triu_indices(n, 1)
    np.testing.assert_allclose(lam.sum(), (D[iu] ** 2).sum() / n, rtol=1e-10)


def test_pcoa_centring_matches_sums():
    """The double centring equals A - row means - column means + grand mean."""
    from oracle import pcoa
    rng = np.random.default_rng(6)
    n = 17
    M = rng.random((n, n))
    D = M + M.T
    np.fill_diagonal(D, 0.0)
    A = -0.5 * D ** 2
    r = A.mean(axis=1)
    want = A - r[:, None] - r[None, :] + A.mean()
    np.testing.assert_allclose(pcoa.double_centred(D), want, atol=1e-12)


# ------------------------------------------------------------------ Mantel oracle

def test_mantel_statistics_match_scipy():
    from scipy import stats as sst
    from oracle import mantel as om
    rng = np.random.default_rng(11)
    x = rng.random(300)
    y = 0.5 * x + rng.random(300)
    np.testing.assert_allclose(om.pearson(x, y), sst.pearsonr(x, y)[0], rtol=1e-12)
    yt = np.round(y * 5) / 5  # ties
    r_s = om.pearson(om.average_ranks(x), om.average_ranks(yt))
    np.testing.assert_allclose(r_s, sst.spearmanr(x, yt)[0], rtol=1e-12)


def test_mantel_permutation_matches_full_matrix():
    """Relabelling the samples of the condensed vector equals permuting the
    rows and columns of the full matrix; the identity changes nothing."""
    from scipy.spatial.distance import squareform
    from oracle import mantel as om
    rng = np.random.default_rng(12)
    n = 9
    y = rng.random(n * (n - 1) // 2)
    perm = rng.permutation(n)
    Y = squareform(y)
    np.testing.assert_array_equal(om.permute_condensed(y, perm, n),
                                  squareform(Y[np.ix_(perm, perm)], checks=False))
    np.testing.assert_array_equal(om.permute_condensed(y, np.arange(n), n), y)


def test_mantel_exhaustive_small_case():
    """n = 4 with all 24 relabellings: y is x relabelled by a known
    permutation, so exactly the permutations giving back x reach r = 1."""
    import itertools
    from oracle import mantel as om
    rng = np.random.default_rng(13)
    n = 4
    x = rng.random(6)
    sigma = np.array([2, 0, 3, 1])
    y = om.permute_condensed(x, sigma, n)
    perms = np.array(list(itertools.permutations(range(n))))
    r, stats, p = om.mantel(x, y, n, perms)
    hits = [q for q, s in zip(perms, stats) if abs(s - 1.0) < 1e-12]
    for q in hits:  # relabelling y by q gives x back
        np.testing.assert_allclose(om.permute_condensed(y, q, n), x)
    assert len(hits) >= 1
    assert 0.0 < p <= 1.0


def test_mantel_p_value_is_two_sided():
    """With n = 3 the three pairs are (0,1), (0,2), (1,2); relabelling the
    samples by pi sends the pair without sample c to the pair without pi(c),
    so the six permutations realise all six orders of the pair vector.  For
    x = y = (1, 2, 3) the statistics are the Pearson correlations of (1, 2, 3)
    with its six orders, which are 1, 1/2, 1/2, -1/2, -1/2, -1 (the sample
    reversal gives -1).  A two-sided count |r_m| >= |r| = 1 takes the identity
    and the reversal: p = 3/7.  The one-sided counts r_m >= r and r_m <= r
    would give 2/7; for y = reversed x (r = -1) the one-sided count r_m >= r
    would give 7/7, the two-sided one 3/7 again."""
    import itertools
    from oracle import mantel as om
    n = 3
    x = np.array([1.0, 2.0, 3.0])
    perms = np.array(list(itertools.permutations(range(n))))
    r, stats, p = om.mantel(x, x.copy(), n, perms)
    assert r == 1.0
    assert sorted(stats.tolist()) == pytest.approx([-1.0, -0.5, -0.5, 0.5, 0.5, 1.0], abs=1e-15)
    rev = [k for k, q in enumerate(perms) if list(q) == [2, 1, 0]][0]
    assert stats[rev] == pytest.approx(-1.0, abs=1e-15)
    assert p == pytest.approx(3.0 / 7.0, abs=1e-15)
    r, stats, p = om.mantel(x, x[::-1].copy(), n, perms)
    assert r == pytest.approx(-1.0, abs=1e-15)
    assert p == pytest.approx(3.0 / 7.0, abs=1e-15)
    # without the reversal only the identity reaches |r|: p = 2/(M + 1)
    r, stats, p = om.mantel(x, x.copy(), n, perms[[k for k in range(6) if k != rev]])
    assert p == pytest.approx(2.0 / 6.0, abs=1e-15)


def test_mantel_undefined_cases():
    """A constant matrix has no correlation (r, r_m and p NaN); without
    permutations there is no null distribution (p NaN, r still defined); the
    p-value counts the identity as one of the M + 1 relabellings."""
    from oracle import mantel as om
    rng = np.random.default_rng(14)
    n = 6
    x = rng.random(15)
    perms = np.array([rng.permutation(n) for _ in range(5)])
    r, stats, p = om.mantel(x, np.full(15, 0.5), n, perms)
    assert np.isnan(r) and np.isnan(p) and np.isnan(stats).all()
    r, stats, p = om.mantel(x, x, n, perms[:0])
    assert r == pytest.approx(1.0, abs=1e-15) and np.isnan(p) and stats.shape == (0,)
    # y = x: each r_m is at most 1 = r, and the identity relabelling reaches it
    ident = np.tile(np.arange(n), (3, 1))
    r, stats, p = om.mantel(x, x, n, ident)
    assert p == 1.0 and np.allclose(stats, 1.0)
