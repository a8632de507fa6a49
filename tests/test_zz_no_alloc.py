"""The allocation-free entry point against the regular one.

unifrac_dense_noalloc serves callers that cannot allocate device memory (its
work space is a fixed array inside the library).  Collected last on purpose:
it calls the entry point twice in a row and compares each result with
unifrac_create + unifrac_run on the same problem, within the FP64 tolerance
the other parity tests use (1e-12).
"""
import ctypes

import numpy as np
import pytest

from paper_2107_05397_b300 import binding as ub
from paper_2107_05397_b300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _noalloc_fn():
    lib = ub.load()
    fn = lib.unifrac_dense_noalloc
    vp = ctypes.c_void_p
    fn.argtypes = [ctypes.c_int, ctypes.c_int32, vp, vp, ctypes.c_int32, vp, vp, vp]
    fn.restype = ctypes.c_int
    return fn


@pytest.mark.parametrize("variant", [ub.UNWEIGHTED, ub.WEIGHTED_NORMALIZED])
def test_noalloc_matches_regular_entry_point_twice(variant):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    w = synth.make_workload("tips1024_samples256", n_samples=200)
    tree, table = w.tree, w.table
    n, N = tree.n_nodes, table.n_samples
    # regular path
    with ub.Context(tree, table) as ctx:
        ref = ctx.run(variant, ub.FP64, ub.OUT_FULL)
        torch.cuda.synchronize()
        ref = ref.cpu().numpy().reshape(N, N)
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


def test_noalloc_rejects_oversized_problem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fn = _noalloc_fn()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = fn(ub.UNWEIGHTED, 1 << 20, dummy.data_ptr(), dummy.data_ptr(), 8, dummy.data_ptr(),
            dummy.data_ptr(), 0)
    assert rc == -9
