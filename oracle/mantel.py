"""FP64 CPU oracle for the Mantel test between two distance matrices.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark to check the
GPU Mantel test; the product library never imports or calls anything here.

The paper (its Mantel section) correlates two distance matrices and
assesses the correlation by permutation.  Written out from the definition:
for condensed distance vectors x and y over the pairs i < j of n samples,

    r = sum (x - mean x)(y - mean y) / sqrt(sum (x - mean x)^2 sum (y - mean y)^2)

(Pearson; Spearman is Pearson on the average ranks of x and of y).  A
permutation pi of the samples relabels the second matrix,
y_pi(i, j) = y(pi(i), pi(j)); with permutations pi_1 .. pi_M the two-sided
p-value is (1 + #{m : |r_m| >= |r|}) / (M + 1).  Permutations are inputs, so
the GPU test and this oracle use the same ones.  Where the statistic is
undefined (a constant matrix: zero variance) r, every r_m and p are NaN, and
with no permutations p is NaN (there is no null distribution).  Parity pinned: Pearson and
Spearman against scipy, permutation of condensed vectors against permuting
the full matrix, the identity permutation, an exhaustive small case.
"""
from __future__ import annotations

import numpy as np


def condensed_index(i: np.ndarray, j: np.ndarray, n: int) -> np.ndarray:
    """Index of pair (i, j), i != j, in the row-major upper triangle."""
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    return lo * n - lo * (lo + 1) // 2 + (hi - lo - 1)


def permute_condensed(y: np.ndarray, perm: np.ndarray, n: int) -> np.ndarray:
    """Condensed vector of the matrix with samples relabelled by perm."""
    i, j = np.triu_indices(n, 1)
    return np.asarray(y, dtype=np.float64)[condensed_index(perm[i], perm[j], n)]


def average_ranks(v: np.ndarray) -> np.ndarray:
    """1-based ranks, ties sharing the mean of their positions."""
    v = np.asarray(v, dtype=np.float64)
    order = np.argsort(v, kind="stable")
    ranks = np.empty(v.shape[0], dtype=np.float64)
    sv = v[order]
    start = 0
    while start < sv.shape[0]:
        end = start
        while end + 1 < sv.shape[0] and sv[end + 1] == sv[start]:
            end += 1
        ranks[order[start:end + 1]] = 0.5 * (start + end) + 1.0
        start = end + 1
    return ranks


def pearson(x: np.ndarray, y: np.ndarray) -> float:
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    dx, dy = x - x.mean(), y - y.mean()
    norm = np.sqrt((dx * dx).sum() * (dy * dy).sum())
    return float((dx * dy).sum() / norm) if norm > 0 else float("nan")


def mantel(x: np.ndarray, y: np.ndarray, n: int, perms: np.ndarray,
           method: str = "pearson") -> tuple[float, np.ndarray, float]:
    """(r, permuted statistics [M], two-sided p-value)."""
    if method == "spearman":
        x, y = average_ranks(x), average_ranks(y)
    r = pearson(x, y)
    stats = np.array([pearson(x, permute_condensed(y, p, n)) for p in perms], dtype=np.float64)
    if np.isnan(r) or len(perms) == 0:
        return r, stats, float("nan")
    p = (1.0 + np.count_nonzero(np.abs(stats) >= abs(r))) / (len(perms) + 1.0)
    return r, stats, p
