"""The allocation-free entry point against the FP64 oracle and the regular one.

unifrac_dense_noalloc serves callers that cannot allocate device memory (its
work space is a fixed array inside the library).  Collected last on purpose:
it calls the entry point twice in a row and compares each result element by
element with the FP64 oracle and with unifrac_create + unifrac_run on the same
problem, within the FP64 tolerance the other parity tests use (1e-12).  The
cases include an all-zero sample (zero denominators), the largest problem the
fixed work space holds (n_nodes x n_samples = UNIFRAC_NOALLOC_MAX_CELLS with
n_samples = UNIFRAC_NOALLOC_MAX_SAMPLES) and problems just beyond each limit,
which are refused with UNIFRAC_E_UNSUPPORTED.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2107_05397_b300 import binding as ub
from paper_2107_05397_b300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12
MAX_CELLS = 1 << 20
MAX_SAMPLES = 4096
E_UNSUPPORTED = -9


def _noalloc_fn():
    lib = ub.load()
    fn = lib.unifrac_dense_noalloc
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int, ctypes.c_int32, vp, vp, ctypes.c_int32, vp, vp, vp]
    fn.restype = ctypes.c_int
    return fn


def _cases():
    """(name, tree, table) of the compared problems."""
    w = synth.make_workload("tips1024_samples256", n_samples=200)
    out = [("workload", w.tree, w.table)]
    # a general tree of exactly 256 nodes and 4,096 samples: the cell limit;
    # samples 0 and 4,095 hold no counts
    rng = np.random.default_rng(41)
    tree = synth.random_general_tree(256, rng, max_children=4, zero_length_prob=0.05)
    tips = tree.tips()
    dense = (rng.random((tips.shape[0], MAX_SAMPLES)) < 0.1) * \
        rng.integers(1, 50, (tips.shape[0], MAX_SAMPLES))
    dense[:, [0, MAX_SAMPLES - 1]] = 0
    out.append(("cell_limit", tree, synth.dense_to_table(dense, rng.permutation(tips))))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", range(len(CASES)), ids=[c[0] for c in CASES])
@pytest.mark.parametrize("variant", [ub.UNWEIGHTED, ub.WEIGHTED_NORMALIZED])
def test_noalloc_matches_oracle_and_regular_entry_point_twice(variant, case):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _, tree, table = CASES[case]
    n, N = tree.n_nodes, table.n_samples
    assert n * N <= MAX_CELLS and N <= MAX_SAMPLES
    ref = oracle.unifrac_full(tree, table, variant)
    # regular path
    with ub.Context(tree, table) as ctx:
        reg = ctx.run(variant, ub.FP64, ub.OUT_FULL)
        torch.cuda.synchronize()
        reg = reg.cpu().numpy().reshape(N, N)
    assert np.max(np.abs(reg - ref)) <= TOL
    # inputs of the allocation-free call, prepared by the caller
    tips = np.zeros((n, N), dtype=np.uint32)
    tips[table.feature_node] = table.dense().astype(np.uint32)
    d_parent = torch.from_numpy(tree.parent.astype(np.int32)).cuda()
    d_length = torch.from_numpy(tree.length.astype(np.float64)).cuda()
    d_tips = torch.from_numpy(tips.view(np.int32)).cuda()
    out = torch.full((N, N), -1.0, dtype=torch.float64, device="cuda")
    fn = _noalloc_fn()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(-1.0)
        rc = fn(variant, n, d_parent.data_ptr(), d_length.data_ptr(), N, d_tips.data_ptr(),
                out.data_ptr(), stream)
        assert rc == 0, ub.unifrac_strerror(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= TOL
        assert np.max(np.abs(got - reg)) <= TOL
        assert np.all(np.diag(got) == 0.0)


def test_noalloc_rejects_problems_beyond_its_work_space():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fn = _noalloc_fn()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    # one cell row over the limit (257 nodes x 4,081 samples), far over it, and
    # one sample over the sample limit with few nodes
    for n_nodes, n_samples in ((257, 4081), (1 << 20, 8), (3, MAX_SAMPLES + 1)):
        assert n_nodes * n_samples > MAX_CELLS or n_samples > MAX_SAMPLES
        rc = fn(ub.UNWEIGHTED, n_nodes, p, p, n_samples, p, p, 0)
        assert rc == E_UNSUPPORTED
