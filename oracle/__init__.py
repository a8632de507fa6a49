"""FP64 CPU oracle for the all-pairs UniFrac distance matrix (ctypes loader).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the benchmark's ``cpu_baseline`` / ``--impl reference`` legs.  The
product library never imports, links or calls anything here.

The arithmetic lives in ``unifrac_oracle.c`` (plain C, FP64, OpenMP over
columns); this module compiles it with gcc on first use and marshals numpy
arrays.  See that file's header for the definitions it follows (paper,
Section II, with the standard unweighted / weighted-normalized formulas).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "unifrac_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None

UNWEIGHTED = 0
WEIGHTED_NORMALIZED = 1


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            f64p = ctypes.POINTER(ctypes.c_double)
            u8p = ctypes.POINTER(ctypes.c_ubyte)
            common = [ctypes.c_int32, i32p, f64p, ctypes.c_int32, i32p, ctypes.c_int32,
                      i64p, i32p, i32p]
            lib.oracle_embedding.argtypes = common + [ctypes.c_int32, f64p, u8p]
            lib.oracle_embedding.restype = ctypes.c_int
            lib.oracle_unifrac_rows.argtypes = common + [ctypes.c_int, ctypes.c_int32, i32p,
                                                         f64p, ctypes.c_int, i32p]
            lib.oracle_unifrac_rows.restype = ctypes.c_int
            lib.oracle_unifrac_pairs.argtypes = common + [ctypes.c_int, ctypes.c_int64, i32p,
                                                          i32p, f64p]
            lib.oracle_unifrac_pairs.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _common(tree, table):
    parent = np.ascontiguousarray(tree.parent, dtype=np.int32)
    length = np.ascontiguousarray(tree.length, dtype=np.float64)
    fnode = np.ascontiguousarray(table.feature_node, dtype=np.int32)
    indptr = np.ascontiguousarray(table.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(table.indices, dtype=np.int32)
    counts = np.ascontiguousarray(table.counts, dtype=np.int32)
    keep = (parent, length, fnode, indptr, indices, counts)
    args = [ctypes.c_int32(parent.shape[0]), _ptr(parent, ctypes.c_int32),
            _ptr(length, ctypes.c_double), ctypes.c_int32(table.n_features),
            _ptr(fnode, ctypes.c_int32), ctypes.c_int32(table.n_samples),
            _ptr(indptr, ctypes.c_int64), _ptr(indices, ctypes.c_int32),
            _ptr(counts, ctypes.c_int32)]
    return keep, args


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def embedding(tree, table, sample: int) -> tuple[np.ndarray, np.ndarray]:
    """(w, p) for one sample over every node: relative abundance and presence."""
    lib = _load()
    keep, args = _common(tree, table)
    n = tree.parent.shape[0]
    w = np.zeros(n, dtype=np.float64)
    p = np.zeros(n, dtype=np.uint8)
    _check(lib.oracle_embedding(*args, ctypes.c_int32(sample), _ptr(w, ctypes.c_double),
                                _ptr(p, ctypes.c_ubyte)), "embedding")
    del keep
    return w, p


def unifrac_rows(tree, table, variant: int, rows: Sequence[int],
                 n_threads: int = 0) -> tuple[np.ndarray, int]:
    """d(rows[r], j) for every j: float64 [len(rows), N] and the thread count."""
    lib = _load()
    keep, args = _common(tree, table)
    rows_a = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
    out = np.zeros((rows_a.shape[0], table.n_samples), dtype=np.float64)
    used = ctypes.c_int32(0)
    _check(lib.oracle_unifrac_rows(*args, ctypes.c_int(variant), ctypes.c_int32(rows_a.shape[0]),
                                   _ptr(rows_a, ctypes.c_int32), _ptr(out, ctypes.c_double),
                                   ctypes.c_int(n_threads), ctypes.byref(used)), "rows")
    del keep
    return out, int(used.value)


def unifrac_full(tree, table, variant: int, n_threads: int = 0) -> np.ndarray:
    """The whole N x N matrix (small cases)."""
    out, _ = unifrac_rows(tree, table, variant, np.arange(table.n_samples), n_threads)
    return out


def unifrac_pairs(tree, table, variant: int, pi: Sequence[int],
                  pj: Sequence[int]) -> np.ndarray:
    """d(pi[k], pj[k]) for an explicit pair list."""
    lib = _load()
    keep, args = _common(tree, table)
    a = np.ascontiguousarray(np.asarray(pi, dtype=np.int32))
    b = np.ascontiguousarray(np.asarray(pj, dtype=np.int32))
    out = np.zeros(a.shape[0], dtype=np.float64)
    _check(lib.oracle_unifrac_pairs(*args, ctypes.c_int(variant), ctypes.c_int64(a.shape[0]),
                                    _ptr(a, ctypes.c_int32), _ptr(b, ctypes.c_int32),
                                    _ptr(out, ctypes.c_double)), "pairs")
    del keep
    return out
