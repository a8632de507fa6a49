"""GPU parity on degenerate problems, through the C ABI, against the FP64
oracle (and, for the three-node tree, against the distances worked out by
hand from the definitions of Section II):

* a tree of one node (the root, which is also the only tip);
* a tree whose branches all have length zero, so no branch is kept;
* samples that are all identical;
* a three-node tree (two tips under the root) with one sample on each tip
  and one on both;
* a context with no samples.

Tolerances as in every other parity test: 1e-12 (FP64), 2e-6 (mixed).
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


def _matrices(tree, table, precision):
    """Both variants' full matrices from one UNIFRAC_BOTH call and from two
    single-variant calls (FP64 numpy, [2, N, N] each)."""
    import torch
    N = table.n_samples
    with ub.Context(tree, table) as ctx:
        both = ctx.run(ub.BOTH, precision, ub.OUT_FULL)
        one = [ctx.run(v, precision, ub.OUT_FULL) for v in VARIANTS]
        torch.cuda.synchronize()
        both = both.cpu().numpy().astype(np.float64).reshape(2, N, N)
        one = np.stack([o.cpu().numpy().astype(np.float64).reshape(N, N) for o in one])
    return both, one


def _check(tree, table, expect=None):
    refs = np.stack([oracle.unifrac_full(tree, table, v) for v in VARIANTS])
    if expect is not None:
        assert np.max(np.abs(refs - expect)) <= 1e-15
    for p in PRECISIONS:
        both, one = _matrices(tree, table, p)
        np.testing.assert_array_equal(both, one)
        assert np.max(np.abs(one - refs)) <= TOL[p], p


def test_one_node_tree():
    """The root is the only node and the only tip: no branch counts, every
    distance is 0."""
    tree = synth.Tree(parent=np.array([-1], np.int32), length=np.array([0.5]))
    table = synth.dense_to_table(np.array([[3, 0, 1, 7]]), np.array([0], np.int32))
    _check(tree, table, expect=np.zeros((2, 4, 4)))


def test_all_branch_lengths_zero():
    """No branch has a length, so none is kept: every distance is 0."""
    rng = np.random.default_rng(21)
    tree, table = synth.random_case(rng, 40, 70, density=0.3, empty_samples=2)
    tree.length[:] = 0.0
    _check(tree, table, expect=np.zeros((2, 70, 70)))


def test_identical_samples():
    """Samples with the same counts (and one with the same proportions at
    twice the counts) are at distance 0 from each other."""
    rng = np.random.default_rng(22)
    tree, _ = synth.random_case(rng, 50, 1)
    tips = tree.tips().astype(np.int32)
    dense = np.zeros((tips.shape[0], 140), np.int64)
    dense[[1, 4, 7, 30], :] = np.array([2, 5, 1, 9])[:, None]
    dense[:, 139] *= 2
    table = synth.dense_to_table(dense, tips)
    _check(tree, table, expect=np.zeros((2, 140, 140)))


def test_three_node_tree_closed_form():
    """Two tips of lengths a and b under the root; sample 0 on tip 0, sample 1
    on tip 1, sample 2 with counts 1 and 3 on both.  From the definitions:
    unweighted d01 = 1, d02 = b / (a + b), d12 = a / (a + b); weighted
    d01 = 1, d02 = (3a/4 + 3b/4) / (5a/4 + 3b/4),
    d12 = (a/4 + b/4) / (a/4 + 7b/4)."""
    a, b = 0.3, 1.7
    tree = synth.Tree(parent=np.array([2, 2, -1], np.int32), length=np.array([a, b, 0.0]))
    table = synth.dense_to_table(np.array([[2, 0, 1], [0, 5, 3]]), np.array([0, 1], np.int32))
    uw = np.array([[0, 1, b / (a + b)], [1, 0, a / (a + b)], [b / (a + b), a / (a + b), 0]])
    w02 = (0.75 * a + 0.75 * b) / (1.25 * a + 0.75 * b)
    w12 = (0.25 * a + 0.25 * b) / (0.25 * a + 1.75 * b)
    wn = np.array([[0, 1, w02], [1, 0, w12], [w02, w12, 0]])
    _check(tree, table, expect=np.stack([uw, wn]))


def test_no_samples():
    """A context over zero samples has empty outputs, and runs into them
    succeed in every layout."""
    rng = np.random.default_rng(23)
    tree, _ = synth.random_case(rng, 10, 1)
    tips = tree.tips().astype(np.int32)
    table = synth.dense_to_table(np.zeros((tips.shape[0], 0), np.int64), tips)
    with ub.Context(tree, table) as ctx:
        for p in PRECISIONS:
            for layout in (ub.OUT_CONDENSED, ub.OUT_FULL, ub.OUT_STRIPES):
                assert ctx.output_bytes(p, layout) == 0
                out = ctx.run(ub.BOTH, p, layout)
                assert out.numel() == 0
