"""Seeded synthetic inputs shaped like the paper's microbiome workloads.

This module holds input generators only: random rooted trees, branch lengths
and sparse feature x sample count tables.  It contains none of the UniFrac
arithmetic, so both the FP64 oracle (tests) and the CUDA path (bench, tests)
draw their inputs from here without sharing any of the method.

The paper (Section II) motivates the shapes: tens of thousands of samples, a
phylogenetic tree over the observed features, and very sparse tables (a given
microbe is absent from the great majority of samples).  The Earth Microbiome
Project data it cites is not available, so these seeded generators stand in.

Conventions shared with the C ABI:
  * tree nodes are numbered in postorder, the root is node n-1 and
    parent[k] > k for every k < n-1, parent[n-1] = -1;
  * length[k] is the length of the branch above node k (root length 0);
  * the table is CSR with one row per feature and column = sample id;
    feature_node[f] is the tip node that feature f sits on.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import os
from typing import Optional

import numpy as np

SEED_BASE = 210705397


@dataclasses.dataclass
class Tree:
    parent: np.ndarray  # int32[n]
    length: np.ndarray  # float64[n]

    @property
    def n_nodes(self) -> int:
        return int(self.parent.shape[0])

    def tips(self) -> np.ndarray:
        """Nodes with no children, ascending."""
        has_child = np.zeros(self.n_nodes, dtype=bool)
        p = self.parent[:-1]
        has_child[p[p >= 0]] = True
        return np.nonzero(~has_child)[0].astype(np.int32)


@dataclasses.dataclass
class Table:
    n_features: int
    n_samples: int
    indptr: np.ndarray  # int64[F+1]
    indices: np.ndarray  # int32[nnz] sample ids
    counts: np.ndarray  # int32[nnz]
    feature_node: np.ndarray  # int32[F]
    study_offsets: Optional[np.ndarray] = None  # int32[S+1] or None

    @property
    def nnz(self) -> int:
        return int(self.indices.shape[0])

    def dense(self) -> np.ndarray:
        """Dense int64 [F, N] copy (small cases only)."""
        out = np.zeros((self.n_features, self.n_samples), dtype=np.int64)
        rows = np.repeat(np.arange(self.n_features), np.diff(self.indptr))
        out[rows, self.indices] = self.counts
        return out


# ----------------------------------------------------------------------------
# trees


def postorder_relabel(children_left: np.ndarray, children_right: np.ndarray,
                      old_parent: np.ndarray, root: int,
                      lengths_old: np.ndarray) -> Tree:
    """Relabel a binary tree given by child arrays into postorder numbering."""
    n = old_parent.shape[0]
    order = np.empty(n, dtype=np.int64)
    stack = [root]
    k = 0
    left = children_left
    right = children_right
    while stack:
        v = stack.pop()
        order[k] = v
        k += 1
        lc = left[v]
        if lc >= 0:
            stack.append(int(lc))
            stack.append(int(right[v]))
    assert k == n
    post = order[::-1]  # left subtree, right subtree, node
    new_id = np.empty(n, dtype=np.int64)
    new_id[post] = np.arange(n)
    parent = np.full(n, -1, dtype=np.int32)
    op = old_parent[post]
    mask = op >= 0
    parent[mask] = new_id[op[mask]].astype(np.int32)
    length = lengths_old[post].astype(np.float64)
    length[-1] = 0.0
    return Tree(parent=parent, length=length)


def yule_tree(n_tips: int, rng: np.random.Generator, mean_length: float) -> Tree:
    """Yule (pure-birth) binary tree: repeatedly split a uniformly chosen tip.

    Branch lengths are Exp(mean_length), the root branch has length 0.
    """
    if n_tips < 1:
        raise ValueError("n_tips must be >= 1")
    n = 2 * n_tips - 1
    left = np.full(n, -1, dtype=np.int64)
    right = np.full(n, -1, dtype=np.int64)
    parent = np.full(n, -1, dtype=np.int64)
    leaves = [0]
    nxt = 1
    u = rng.random(max(n_tips - 1, 0))
    for step in range(n_tips - 1):
        r = int(u[step] * len(leaves))
        v = leaves[r]
        a, b = nxt, nxt + 1
        nxt += 2
        left[v], right[v] = a, b
        parent[a] = v
        parent[b] = v
        leaves[r] = a
        leaves.append(b)
    lengths = rng.exponential(mean_length, size=n)
    return postorder_relabel(left, right, parent, 0, lengths)


def star_tree(n_tips: int, branch_length: float = 1.0) -> Tree:
    """Root with n_tips children, every tip branch the same length."""
    parent = np.full(n_tips + 1, n_tips, dtype=np.int32)
    parent[-1] = -1
    length = np.full(n_tips + 1, branch_length, dtype=np.float64)
    length[-1] = 0.0
    return Tree(parent=parent, length=length)


def random_general_tree(n_nodes: int, rng: np.random.Generator,
                        max_children: int = 4, mean_length: float = 0.5,
                        zero_length_prob: float = 0.0) -> Tree:
    """Random rooted tree with multifurcations and unary nodes, postorder.

    Built top-down: node k (k < n-1) gets a parent chosen uniformly among the
    nodes above it in the final numbering whose child count is below
    max_children, so parent[k] > k always holds.
    """
    if n_nodes < 1:
        raise ValueError("n_nodes must be >= 1")
    parent = np.full(n_nodes, -1, dtype=np.int32)
    nchild = np.zeros(n_nodes, dtype=np.int64)
    for k in range(n_nodes - 2, -1, -1):
        cands = np.arange(k + 1, n_nodes)
        cands = cands[nchild[cands] < max_children]
        p = int(cands[rng.integers(cands.shape[0])])
        parent[k] = p
        nchild[p] += 1
    length = rng.exponential(mean_length, size=n_nodes)
    if zero_length_prob > 0:
        length[rng.random(n_nodes) < zero_length_prob] = 0.0
    length[-1] = 0.0
    # This numbering is a valid topological order (children before parents);
    # convert it to a true postorder so subtrees are contiguous ranges.
    return to_postorder(parent, length)


def to_postorder(parent: np.ndarray, length: np.ndarray) -> Tree:
    """Renumber any rooted tree (parent array, one root) into postorder."""
    n = parent.shape[0]
    roots = np.nonzero(parent < 0)[0]
    assert roots.shape[0] == 1
    kids: list[list[int]] = [[] for _ in range(n)]
    for v in range(n):
        if parent[v] >= 0:
            kids[int(parent[v])].append(v)
    order = []
    stack = [(int(roots[0]), 0)]
    while stack:
        v, i = stack.pop()
        if i < len(kids[v]):
            stack.append((v, i + 1))
            stack.append((kids[v][i], 0))
        else:
            order.append(v)
    post = np.asarray(order, dtype=np.int64)
    new_id = np.empty(n, dtype=np.int64)
    new_id[post] = np.arange(n)
    p_new = np.full(n, -1, dtype=np.int32)
    op = parent[post]
    m = op >= 0
    p_new[m] = new_id[op[m]].astype(np.int32)
    l_new = np.asarray(length, dtype=np.float64)[post].copy()
    l_new[-1] = 0.0
    return Tree(parent=p_new, length=l_new)


# ----------------------------------------------------------------------------
# tables


def _draw_features(rng: np.random.Generator, cdf: Optional[np.ndarray],
                   n_features: int, k: int) -> np.ndarray:
    """k distinct features by successive weighted sampling without replacement.

    Drawing with replacement and keeping first occurrences in draw order is the
    same distribution as drawing one at a time without replacement.
    """
    if cdf is None:
        return rng.choice(n_features, size=k, replace=False)
    got: list[np.ndarray] = []
    seen = np.empty(0, dtype=np.int64)
    while True:
        m = 2 * k + 64
        u = rng.random(m) * cdf[-1]
        # inverse CDF; the needles are searched in sorted order (same result,
        # fewer cache misses on a large cdf)
        order = np.argsort(u)
        draw = np.empty(m, dtype=np.int64)
        draw[order] = np.searchsorted(cdf, u[order], side="right")
        draw = np.minimum(draw, n_features - 1)
        cat = np.concatenate([seen, draw])
        _, first = np.unique(cat, return_index=True)
        first.sort()
        seen = cat[first]
        if seen.shape[0] >= k:
            return seen[:k]
        got.append(draw)


def synth_table(tree: Tree, n_samples: int, density: float,
                zipf_s: Optional[float], lognorm_mu: float,
                lognorm_sigma: float, rng: np.random.Generator,
                n_features: Optional[int] = None,
                density_per_sample: Optional[np.ndarray] = None) -> Table:
    """Sparse count table over the tree's tips.

    Per sample: k ~ Binomial(F, density) (at least 1) distinct features, drawn
    with Zipf(s) popularity over a random ranking (uniform if zipf_s is None);
    counts = round(LogNormal(mu, sigma)) + 1.  Features sit on a seeded random
    permutation of the tips.
    """
    tips = tree.tips()
    F = tips.shape[0] if n_features is None else int(n_features)
    if F > tips.shape[0]:
        raise ValueError("more features than tips")
    feature_node = rng.permutation(tips)[:F].astype(np.int32)
    if zipf_s is None:
        cdf = None
    else:
        rank = rng.permutation(F)
        w = (rank.astype(np.float64) + 1.0) ** (-float(zipf_s))
        cdf = np.cumsum(w)
    rows_l, cols_l, vals_l = [], [], []
    for i in range(n_samples):
        d = density if density_per_sample is None else float(density_per_sample[i])
        k = max(1, int(rng.binomial(F, d)))
        k = min(k, F)
        feats = _draw_features(rng, cdf, F, k)
        cnt = np.rint(rng.lognormal(lognorm_mu, lognorm_sigma, size=k)) + 1
        cnt = np.minimum(cnt, 2**31 - 1)
        rows_l.append(feats.astype(np.int64))
        cols_l.append(np.full(k, i, dtype=np.int64))
        vals_l.append(cnt.astype(np.int64))
    return coo_to_table(F, n_samples, np.concatenate(rows_l) if rows_l else np.empty(0, np.int64),
                        np.concatenate(cols_l) if cols_l else np.empty(0, np.int64),
                        np.concatenate(vals_l) if vals_l else np.empty(0, np.int64),
                        feature_node)


def coo_to_table(n_features: int, n_samples: int, rows: np.ndarray,
                 cols: np.ndarray, vals: np.ndarray,
                 feature_node: np.ndarray,
                 study_offsets: Optional[np.ndarray] = None) -> Table:
    """Build a CSR table (rows = features, sorted sample ids) from COO triples."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.int64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    indptr = np.zeros(n_features + 1, dtype=np.int64)
    np.add.at(indptr, rows + 1, 1)
    indptr = np.cumsum(indptr)
    return Table(n_features=n_features, n_samples=n_samples, indptr=indptr,
                 indices=cols.astype(np.int32), counts=vals.astype(np.int32),
                 feature_node=np.asarray(feature_node, dtype=np.int32),
                 study_offsets=None if study_offsets is None
                 else np.asarray(study_offsets, dtype=np.int32))


def dense_to_table(dense: np.ndarray, feature_node: np.ndarray) -> Table:
    """CSR table from a dense [F, N] count matrix (zeros dropped)."""
    dense = np.asarray(dense)
    r, c = np.nonzero(dense)
    return coo_to_table(dense.shape[0], dense.shape[1], r, c, dense[r, c],
                        feature_node)


# ----------------------------------------------------------------------------
# named workloads (sizes as in the paper's discussion of 25k-50k samples)


@dataclasses.dataclass
class Workload:
    name: str
    tree: Tree
    table: Table
    description: str


WORKLOADS = {
    # small: FP64, both variants, full 256 x 256
    "tips1024_samples256": dict(index=1, tips=1024, mean_len=0.1, samples=256,
                                density=0.03, zipf=None, mu=2.0, sigma=1.0),
    # plain FP64 vs mixed on 4,096 samples, condensed output
    "tips32768_samples4096": dict(index=2, tips=32768, mean_len=0.1, samples=4096,
                                  density=0.01, zipf=1.1, mu=2.0, sigma=1.5),
    # EMP-sized: 25k samples on a 200k-tip tree
    "tips200000_samples25000": dict(index=3, tips=200000, mean_len=0.05,
                                    samples=25000, density=0.002, zipf=1.2,
                                    mu=2.0, sigma=1.0),
    # 50k samples on the same 200k-tip tree
    "tips200000_samples50000": dict(index=4, tips=200000, mean_len=0.05,
                                    samples=50000, density=0.002, zipf=1.2,
                                    mu=2.0, sigma=1.0, tree_index=3),
}

BATCHED = {
    "tips50000_studies64": dict(index=5, tips=50000, mean_len=0.05, studies=64,
                                n_lo=200, n_hi=6000, d_lo=0.005, d_hi=0.03,
                                zipf=1.2, mu=2.0, sigma=1.0),
}


def _cache_path(name: str, n_samples: Optional[int]) -> Optional[str]:
    """File of a named workload in the cache directory (environment variable
    UNIFRAC_SYNTH_CACHE, default a folder under the system temp directory;
    "off" disables it), keyed by this module's source so that any change to a
    generator starts a new entry."""
    d = os.environ.get("UNIFRAC_SYNTH_CACHE")
    if d == "off":
        return None
    if not d:
        import tempfile
        d = os.path.join(tempfile.gettempdir(), "unifrac_synth_cache")
    with open(os.path.abspath(__file__), "rb") as f:
        key = hashlib.sha256(f.read()).hexdigest()[:16]
    return os.path.join(d, f"{name}-{n_samples}-{key}.npz")


def _save(path: str, w: Workload) -> None:
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp.npz"
        t = w.table
        np.savez(tmp, parent=w.tree.parent, length=w.tree.length, indptr=t.indptr,
                 indices=t.indices, counts=t.counts, feature_node=t.feature_node,
                 study_offsets=(np.empty(0, np.int32) if t.study_offsets is None
                                else t.study_offsets),
                 meta=np.array([t.n_features, t.n_samples], np.int64),
                 description=np.array(w.description))
        os.replace(tmp, path)
    except OSError:
        pass


def _load(path: str, name: str) -> Optional[Workload]:
    try:
        z = np.load(path)
        so = z["study_offsets"]
        table = Table(n_features=int(z["meta"][0]), n_samples=int(z["meta"][1]),
                      indptr=z["indptr"], indices=z["indices"], counts=z["counts"],
                      feature_node=z["feature_node"],
                      study_offsets=None if so.shape[0] == 0 else so)
        return Workload(name=name, tree=Tree(parent=z["parent"], length=z["length"]),
                        table=table, description=str(z["description"]))
    except (OSError, KeyError, ValueError):
        return None


def make_workload(name: str, n_samples: Optional[int] = None) -> Workload:
    """Build a named seeded workload; n_samples optionally truncates N.  The
    large ones take a minute or more to draw, so they are kept in a cache
    folder (see _cache_path) and read back by later processes."""
    path = _cache_path(name, n_samples)
    if path and os.path.exists(path):
        w = _load(path, name)
        if w is not None:
            return w
    w = _make_workload(name, n_samples)
    if path and w.table.nnz >= 1_000_000:
        _save(path, w)
    return w


def _make_workload(name: str, n_samples: Optional[int] = None) -> Workload:
    if name in BATCHED:
        return make_batched(name)
    p = WORKLOADS[name]
    tree_seed = SEED_BASE + p.get("tree_index", p["index"])
    tree = yule_tree(p["tips"], np.random.default_rng(tree_seed), p["mean_len"])
    rng = np.random.default_rng([SEED_BASE + p["index"], 1])
    N = p["samples"] if n_samples is None else int(n_samples)
    table = synth_table(tree, N, p["density"], p["zipf"], p["mu"], p["sigma"], rng)
    desc = (f"Yule tree {p['tips']} tips Exp({p['mean_len']}) lengths; "
            f"{N} samples at {p['density']*100:g}% density, "
            f"{'uniform' if p['zipf'] is None else 'Zipf(%g)' % p['zipf']} features, "
            f"counts round(LogNormal({p['mu']},{p['sigma']}))+1")
    return Workload(name=name, tree=tree, table=table, description=desc)


def make_batched(name: str, n_studies: Optional[int] = None) -> Workload:
    """Many studies of uneven size sharing one tree (samples concatenated)."""
    p = BATCHED[name]
    tree = yule_tree(p["tips"], np.random.default_rng(SEED_BASE + p["index"]),
                     p["mean_len"])
    rng = np.random.default_rng([SEED_BASE + p["index"], 1])
    S = p["studies"] if n_studies is None else int(n_studies)
    sizes = np.rint(np.exp(rng.uniform(math.log(p["n_lo"]), math.log(p["n_hi"]),
                                       size=S))).astype(np.int64)
    dens = rng.uniform(p["d_lo"], p["d_hi"], size=S)
    per_sample = np.repeat(dens, sizes)
    N = int(sizes.sum())
    table = synth_table(tree, N, 0.0, p["zipf"], p["mu"], p["sigma"], rng,
                        density_per_sample=per_sample)
    offs = np.zeros(S + 1, dtype=np.int32)
    offs[1:] = np.cumsum(sizes)
    table.study_offsets = offs
    desc = (f"{S} studies sharing a Yule tree of {p['tips']} tips; study sizes "
            f"log-uniform {p['n_lo']}-{p['n_hi']} (total {N}), densities "
            f"U({p['d_lo']*100:g}%,{p['d_hi']*100:g}%), Zipf({p['zipf']})")
    return Workload(name=name, tree=tree, table=table, description=desc)


def random_case(rng: np.random.Generator, n_tips: int, n_samples: int,
                density: float = 0.3, general: bool = False,
                empty_samples: int = 0) -> tuple[Tree, Table]:
    """Small random tree + table for parity and property tests."""
    if general:
        tree = random_general_tree(max(2 * n_tips, 2), rng, max_children=4)
    else:
        tree = yule_tree(n_tips, rng, 0.3)
    tips = tree.tips()
    F = tips.shape[0]
    dense = (rng.random((F, n_samples)) < density) * rng.integers(1, 20, size=(F, n_samples))
    if empty_samples:
        cols = rng.choice(n_samples, size=min(empty_samples, n_samples), replace=False)
        dense[:, cols] = 0
    feature_node = rng.permutation(tips).astype(np.int32)
    return tree, dense_to_table(dense, feature_node)
