"""C-ABI checks that need no GPU: the library loads, exports every function
that include/unifrac_b300.h declares, and rejects malformed inputs with the
documented status codes before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2107_05397_b300 import binding as ub
from paper_2107_05397_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "unifrac_b300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(unifrac_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = ub.load()
    names = declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name
    assert set(ub.EXPORTED) <= set(names)


def test_binding_declares_every_entry_point():
    """binding.load() gives every declared function its ctypes signature, so
    no other module has to (or may) set one on the shared library handle."""
    lib = ub.load()
    for name in declared_functions():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name


def test_autotune_rejects_null_context_or_buffer():
    lib = ub.load()
    buf = ctypes.create_string_buffer(16)
    assert lib.unifrac_autotune(None, ub.UNWEIGHTED, ub.MIXED, buf, 16, 2) == -1
    assert lib.unifrac_autotune(None, ub.UNWEIGHTED, ub.MIXED, None, 16, 2) == -1


def test_strerror_covers_codes():
    for code in range(0, -10, -1):
        s = ub.unifrac_strerror(code)
        assert s and s != "unknown status"
    assert ub.unifrac_strerror(-99) == "unknown status"


def _tiny():
    tree = synth.Tree(parent=np.array([2, 2, 4, 4, -1], np.int32),
                      length=np.array([1.0, 2.0, 0.5, 1.5, 0.0]))
    table = synth.dense_to_table(np.array([[1, 0, 3], [2, 1, 0], [0, 4, 1]]),
                                 np.array([0, 1, 3], np.int32))
    return tree, table


def _create(tree, table, **kw):
    args = dict(parent=tree.parent, length=tree.length, feature_node=table.feature_node,
                indptr=table.indptr, indices=table.indices, counts=table.counts,
                n_samples=table.n_samples, study_offsets=table.study_offsets, stream=0)
    args.update(kw)
    return ub.unifrac_create(**args)


@pytest.mark.parametrize("mutate,code", [
    (lambda t, b: dict(parent=np.array([2, 0, 4, 4, -1], np.int32)), -2),   # not postorder
    (lambda t, b: dict(parent=np.array([2, 2, 4, 4, 3], np.int32)), -2),    # root has a parent
    (lambda t, b: dict(length=np.array([1.0, -2.0, 0.5, 1.5, 0.0])), -2),   # negative length
    (lambda t, b: dict(length=np.array([1.0, np.nan, 0.5, 1.5, 0.0])), -2), # NaN length
    (lambda t, b: dict(feature_node=np.array([0, 2, 3], np.int32)), -2),    # internal node
    (lambda t, b: dict(feature_node=np.array([0, 0, 3], np.int32)), -3),    # two features on a tip
    (lambda t, b: dict(feature_node=np.array([0, 1, 7], np.int32)), -2),    # out of range
    (lambda t, b: dict(indices=np.where(b.indices == 2, 5, b.indices).astype(np.int32)), -3),
    (lambda t, b: dict(counts=np.where(np.arange(b.nnz) == 1, -4, b.counts).astype(np.int32)), -3),
    (lambda t, b: dict(study_offsets=np.array([0, 2, 1, 3], np.int32)), -1),
    (lambda t, b: dict(study_offsets=np.array([0, 2], np.int32)), -1),
])
def test_create_rejects_malformed_inputs(mutate, code):
    tree, table = _tiny()
    with pytest.raises(ub.UniFracError) as ei:
        _create(tree, table, **mutate(tree, table))
    assert ei.value.status == code


def test_create_rejects_duplicate_entries():
    tree, table = _tiny()
    indptr = np.array([0, 3, 5, 7], np.int64)
    indices = np.array([0, 0, 2, 0, 1, 1, 2], np.int32)
    counts = np.ones(7, np.int32)
    with pytest.raises(ub.UniFracError) as ei:
        _create(tree, table, indptr=indptr, indices=indices, counts=counts)
    assert ei.value.status == -3


def test_create_rejects_huge_sample_totals():
    tree, _ = _tiny()
    table = synth.dense_to_table(np.array([[1, 1, 3], [2, 1, 0], [0, 4, 1]]),
                                 np.array([0, 1, 3], np.int32))
    counts = np.full(table.nnz, 2**31 - 1, np.int32)
    with pytest.raises(ub.UniFracError) as ei:
        _create(tree, table, counts=counts)
    assert ei.value.status == -3


def test_null_pointers_rejected():
    lib = ub.load()
    out = ctypes.c_void_p()
    assert lib.unifrac_create(5, None, None, 0, None, 0, None, None, None, 1, None, None,
                              ctypes.byref(out)) == -1
    assert lib.unifrac_run(None, 0, 0, 0, -1, 0, None, 0) == -1
    lib.unifrac_destroy(None)
    v = ctypes.c_double()
    assert lib.unifrac_get_stat(None, 0, ctypes.byref(v)) == -1
    assert lib.unifrac_set_option(None, 0, 0) == -1


def test_binding_constants_match_header_enums():
    """Every enumerator of include/unifrac_b300.h has the same value in the
    binding (options, statistics, status codes, variants, precisions,
    layouts), and the binding defines no constant the header lacks."""
    import re
    text = open(os.path.join(os.path.dirname(__file__), "..", "include",
                             "unifrac_b300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    header = {}
    for body in re.findall(r"enum\s+\w*\s*\{(.*?)\}", text, flags=re.S):
        for name, val in re.findall(r"(UNIFRAC_\w+)\s*=\s*(-?\d+)", body):
            header[name] = int(val)
    prefix = {"OPT_": "UNIFRAC_OPT_", "STAT_": "UNIFRAC_STAT_"}
    checked = 0
    for attr in dir(ub):
        for p, hp in prefix.items():
            if attr.startswith(p):
                assert hp + attr[len(p):] in header, attr
                assert getattr(ub, attr) == header[hp + attr[len(p):]], attr
                checked += 1
    for name, val in header.items():
        for hp, p in (("UNIFRAC_OPT_", "OPT_"), ("UNIFRAC_STAT_", "STAT_")):
            if name.startswith(hp):
                assert getattr(ub, p + name[len(hp):]) == val, name
    assert header["UNIFRAC_UNWEIGHTED"] == ub.UNWEIGHTED
    assert header["UNIFRAC_WEIGHTED_NORMALIZED"] == ub.WEIGHTED_NORMALIZED
    assert header["UNIFRAC_BOTH"] == ub.BOTH
    assert header["UNIFRAC_FP64"] == ub.FP64 and header["UNIFRAC_MIXED"] == ub.MIXED
    assert header["UNIFRAC_MANTEL_PEARSON"] == ub.MANTEL_PEARSON
    assert header["UNIFRAC_MANTEL_SPEARMAN"] == ub.MANTEL_SPEARMAN
    m = re.search(r"#define\s+UNIFRAC_MANTEL_MAX_SAMPLES\s+(\d+)", text)
    assert m and int(m.group(1)) == ub.MANTEL_MAX_SAMPLES
    n = ub.MANTEL_MAX_SAMPLES
    assert n * (n - 1) // 2 < 2**32 <= (n + 1) * n // 2  # largest n whose pair indices fit 32 bits
    assert checked >= 25


def test_downstream_bindings_reject_host_tensors_before_the_library():
    """PCoA and the Mantel test take device matrices: host tensors, mixed
    dtypes, non-square sizes and unknown methods are refused in the binding,
    with no library call (no GPU needed)."""
    import torch
    D = torch.zeros((6, 6), dtype=torch.float32)
    with pytest.raises(ValueError):
        ub.unifrac_pcoa(D, k=2)
    with pytest.raises(ValueError):
        ub.unifrac_mantel(D, D, np.tile(np.arange(6, dtype=np.int32), (2, 1)))
    with pytest.raises(ValueError):
        ub.unifrac_mantel(D, D.double(), np.zeros((1, 6), np.int32))


def test_mantel_declaration_matches_binding_argtypes():
    """The ctypes prototype of unifrac_mantel has the header's eleven
    parameters in order (pointer, pointer, int, int32, pointer, int32, int,
    then four pointers)."""
    import ctypes
    lib = ub.load()
    at = lib.unifrac_mantel.argtypes
    assert len(at) == 11
    assert at[2] is ctypes.c_int and at[3] is ctypes.c_int32 and at[5] is ctypes.c_int32
    assert at[6] is ctypes.c_int
    text = open(os.path.join(os.path.dirname(__file__), "..", "include", "unifrac_b300.h")).read()
    decl = text[text.index("int unifrac_mantel("):]
    decl = decl[:decl.index(";")]
    assert decl.count(",") == 10


def test_bounded_wait_check_rejects_bad_limits():
    """Limits outside 1 .. 1,000,000 microseconds are refused before any
    device call."""
    for bad in (0, 1_000_001):
        with pytest.raises(ub.UniFracError) as ei:
            ub.unifrac_check_bounded_wait(bad)
        assert ei.value.status == -1
