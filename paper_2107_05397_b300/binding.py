"""ctypes binding of libunifrac_b300.so: argument marshalling only.

The functions carry the names of the C ABI in ``include/unifrac_b300.h``; every
step of the computation runs in the library's CUDA kernels.  PyTorch is only
used to hand over device buffers and the current CUDA stream.  If the shared
library is missing the binding raises immediately: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libunifrac_b300.so")

UNWEIGHTED = 0
WEIGHTED_NORMALIZED = 1
BOTH = 2
FP64 = 0
MIXED = 1
OUT_STRIPES = 0
OUT_CONDENSED = 1
OUT_FULL = 2

MANTEL_PEARSON = 0
MANTEL_SPEARMAN = 1
MANTEL_MAX_SAMPLES = 92682

OPT_UNWEIGHTED_MIXED_KERNEL = 0
OPT_WEIGHTED_FLUSH = 1
OPT_USE_GRAPH = 4
OPT_SPARSE_THRESHOLD = 5
OPT_UNWEIGHTED_SPARSE_THRESHOLD = 6
OPT_OVERLAP_VARIANTS = 7
OPT_SPARSE_LANE_PAIRS = 8
OPT_UNWEIGHTED_SPARSE_LANE_PAIRS = 9
OPT_PERSISTENT = 10
OPT_RARE_LIST = 11
OPT_UNWEIGHTED_RARE_LIST = 12
OPT_COPY_RANGES = 13
OPT_HOST_THREADS = 14

STAT_KERNEL_LAUNCHES = 0
STAT_PAIR_BRANCH = 1
STAT_USEFUL = 2
STAT_BRANCHES_KEPT = 3
STAT_LEVELS = 4
STAT_TILE_PAIRS = 5
STAT_SELECTED_UPDATES = 6
STAT_PAIR_KERNEL_MS = 7
STAT_EMBED_MS = 8
STAT_DEVICE_BYTES = 9
STAT_PAIR_MS_UNWEIGHTED = 10
STAT_PAIR_MS_WEIGHTED = 11
STAT_DEVICE_ERROR = 12
STAT_SELECTED_UNWEIGHTED = 13
STAT_SELECTED_WEIGHTED = 14
STAT_SPARSE_MS_UNWEIGHTED = 15
STAT_SPARSE_MS_WEIGHTED = 16
STAT_SPARSE_UPDATES_UNWEIGHTED = 17
STAT_SPARSE_UPDATES_WEIGHTED = 18
STAT_CREATE_HOST_MS = 19
STAT_CREATE_DEVICE_MS = 20
STAT_MAX_REACH = 21
STAT_LIST_MS_UNWEIGHTED = 22
STAT_LIST_MS_WEIGHTED = 23
STAT_LIST_UPDATES_UNWEIGHTED = 24
STAT_LIST_UPDATES_WEIGHTED = 25

EXPORTED = ("unifrac_create", "unifrac_run", "unifrac_destroy", "unifrac_strerror",
            "unifrac_last_error", "unifrac_n_stripes", "unifrac_output_bytes",
            "unifrac_set_option", "unifrac_get_option", "unifrac_get_stat",
            "unifrac_autotune", "unifrac_run_streamed", "unifrac_pcoa", "unifrac_mantel",
            "unifrac_check_bounded_wait", "unifrac_measure_peak", "unifrac_set_memory_cache",
            "unifrac_release_cached_memory", "unifrac_cached_memory")

PEAK_FP32_FMA = 0
PEAK_FP64_FMA = 1


class UniFracError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


def load() -> ctypes.CDLL:
    """Load the shared library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2107_05397_b300.build` "
                "(there is no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        lib.unifrac_create.argtypes = [i32, vp, vp, i32, vp, i32, vp, vp, vp, i32, vp, vp,
                                       ctypes.POINTER(vp)]
        lib.unifrac_create.restype = ctypes.c_int
        lib.unifrac_run.argtypes = [vp, ctypes.c_int, ctypes.c_int, i32, i32, ctypes.c_int, vp,
                                    ctypes.c_size_t]
        lib.unifrac_run.restype = ctypes.c_int
        lib.unifrac_run_streamed.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp,
                                             ctypes.c_size_t, i32]
        lib.unifrac_run_streamed.restype = ctypes.c_int
        lib.unifrac_pcoa.argtypes = [vp, ctypes.c_int, i32, i32, i32, ctypes.c_uint64, vp, vp, vp]
        lib.unifrac_pcoa.restype = ctypes.c_int
        lib.unifrac_mantel.argtypes = [vp, vp, ctypes.c_int, i32, vp, i32, ctypes.c_int, vp, vp,
                                       vp, vp]
        lib.unifrac_mantel.restype = ctypes.c_int
        lib.unifrac_check_bounded_wait.argtypes = [ctypes.c_uint32, ctypes.POINTER(i32), vp]
        lib.unifrac_check_bounded_wait.restype = ctypes.c_int
        lib.unifrac_measure_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), vp]
        lib.unifrac_measure_peak.restype = ctypes.c_int
        lib.unifrac_destroy.argtypes = [vp]
        lib.unifrac_destroy.restype = None
        lib.unifrac_strerror.argtypes = [ctypes.c_int]
        lib.unifrac_strerror.restype = ctypes.c_char_p
        lib.unifrac_last_error.argtypes = [vp]
        lib.unifrac_last_error.restype = ctypes.c_char_p
        lib.unifrac_n_stripes.argtypes = [vp, i32, ctypes.POINTER(i32)]
        lib.unifrac_n_stripes.restype = ctypes.c_int
        lib.unifrac_output_bytes.argtypes = [vp, ctypes.c_int, ctypes.c_int, i32, i32,
                                             ctypes.POINTER(ctypes.c_size_t)]
        lib.unifrac_output_bytes.restype = ctypes.c_int
        lib.unifrac_set_option.argtypes = [vp, ctypes.c_int, i64]
        lib.unifrac_set_option.restype = ctypes.c_int
        lib.unifrac_get_option.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
        lib.unifrac_get_option.restype = ctypes.c_int
        lib.unifrac_get_stat.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        lib.unifrac_get_stat.restype = ctypes.c_int
        lib.unifrac_set_memory_cache.argtypes = [ctypes.c_int, i64]
        lib.unifrac_set_memory_cache.restype = ctypes.c_int
        lib.unifrac_release_cached_memory.argtypes = [ctypes.c_int]
        lib.unifrac_release_cached_memory.restype = ctypes.c_int
        lib.unifrac_cached_memory.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
        lib.unifrac_cached_memory.restype = ctypes.c_int
        lib.unifrac_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t,
                                         ctypes.c_int]
        lib.unifrac_autotune.restype = ctypes.c_int
        lib.unifrac_dense_noalloc.argtypes = [ctypes.c_int, i32, vp, vp, i32, vp, vp, vp]
        lib.unifrac_dense_noalloc.restype = ctypes.c_int
        _lib = lib
        return lib


def unifrac_strerror(status: int) -> str:
    return load().unifrac_strerror(status).decode()


def unifrac_last_error(ctx) -> str:
    return load().unifrac_last_error(ctx).decode()


def _check(status: int, ctx=None) -> None:
    if status != 0:
        msg = unifrac_strerror(status)
        if ctx:
            detail = unifrac_last_error(ctx)
            if detail:
                msg = f"{msg}: {detail}"
        raise UniFracError(status, msg)


def _arr(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def unifrac_create(parent, length, feature_node, indptr, indices, counts, n_samples: int,
                   study_offsets=None, stream=None):
    """Validate and upload one problem; returns an opaque context handle."""
    lib = load()
    parent = _arr(parent, np.int32)
    length = _arr(length, np.float64)
    feature_node = _arr(feature_node, np.int32)
    indptr = _arr(indptr, np.int64)
    indices = _arr(indices, np.int32)
    counts = _arr(counts, np.int32)
    so = None if study_offsets is None else _arr(study_offsets, np.int32)
    n_studies = 1 if so is None else so.shape[0] - 1
    if parent.shape != length.shape:
        raise ValueError("parent and length differ in size")
    if indptr.shape[0] != feature_node.shape[0] + 1:
        raise ValueError("indptr must have n_features + 1 entries")
    ctx = ctypes.c_void_p()
    status = lib.unifrac_create(parent.shape[0], _ptr(parent), _ptr(length),
                                feature_node.shape[0], _ptr(feature_node), int(n_samples),
                                _ptr(indptr), _ptr(indices), _ptr(counts), n_studies,
                                None if so is None else _ptr(so), _stream_handle(stream),
                                ctypes.byref(ctx))
    _check(status)
    return ctx


def unifrac_output_bytes(ctx, precision: int, layout: int, stripe_start: int = 0,
                         stripe_stop: int = -1) -> int:
    out = ctypes.c_size_t()
    _check(load().unifrac_output_bytes(ctx, precision, layout, stripe_start, stripe_stop,
                                       ctypes.byref(out)), ctx)
    return int(out.value)


def unifrac_n_stripes(ctx, study: int = 0) -> int:
    out = ctypes.c_int32()
    _check(load().unifrac_n_stripes(ctx, study, ctypes.byref(out)), ctx)
    return int(out.value)


def _data_ptr(out) -> tuple[int, int]:
    """(address, capacity in bytes) of a torch tensor or numpy array."""
    if isinstance(out, np.ndarray):
        if not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be contiguous")
        return out.ctypes.data, out.nbytes
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    return out.data_ptr(), out.numel() * out.element_size()


def unifrac_run(ctx, variant: int, precision: int, stripe_start: int, stripe_stop: int,
                layout: int, out) -> None:
    """Compute into `out` (torch CUDA tensor: asynchronous on the context's
    stream; numpy array / CPU tensor: staged, returns when complete)."""
    addr, cap = _data_ptr(out)
    _check(load().unifrac_run(ctx, variant, precision, stripe_start, stripe_stop, layout,
                              ctypes.c_void_p(addr), cap), ctx)


def unifrac_run_streamed(ctx, variant: int, precision: int, layout: int, out,
                         chunk_stripes: int) -> None:
    """The whole matrix into the HOST array `out` (numpy / CPU tensor), in
    chunks of `chunk_stripes` stripes; returns when complete."""
    addr, cap = _data_ptr(out)
    _check(load().unifrac_run_streamed(ctx, variant, precision, layout, ctypes.c_void_p(addr),
                                       cap, int(chunk_stripes)), ctx)


def unifrac_pcoa(dist, k: int, iters: int = 12, seed: int = 0, stream=None):
    """Principal coordinates of the full distance matrix `dist` (torch CUDA
    tensor, n x n or n*n, float32 or float64): (eigenvalues [k], coordinates
    [n, k]) as FP64 numpy arrays."""
    import torch
    if not (isinstance(dist, torch.Tensor) and dist.is_cuda and dist.is_contiguous()):
        raise ValueError("dist must be a contiguous CUDA tensor")
    if dist.dtype not in (torch.float32, torch.float64):
        raise ValueError("dist must be float32 or float64")
    n = int(round(dist.numel() ** 0.5))
    if n * n != dist.numel():
        raise ValueError("dist must hold n x n values")
    precision = FP64 if dist.dtype == torch.float64 else MIXED
    lam = np.zeros(k, np.float64)
    coords = np.zeros((n, k), np.float64)
    status = load().unifrac_pcoa(ctypes.c_void_p(dist.data_ptr()), precision, n, int(k),
                                 int(iters), ctypes.c_uint64(int(seed) & (2**64 - 1)),
                                 lam.ctypes.data_as(ctypes.c_void_p),
                                 coords.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream))
    _check(status)
    return lam, coords


def unifrac_mantel(x, y, perms, method: str = "pearson", stream=None):
    """Mantel test between the full distance matrices `x` and `y` (torch CUDA
    tensors, n x n or n*n, both float32 or both float64) under the caller's
    permutations `perms` (int array [M, n], each row a permutation of
    0 .. n-1): (r, permuted statistics [M] as FP64 numpy, two-sided p)."""
    import torch
    for t in (x, y):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
            raise ValueError("x and y must be contiguous CUDA tensors")
    if x.dtype != y.dtype or x.dtype not in (torch.float32, torch.float64):
        raise ValueError("x and y must both be float32 or both float64")
    n = int(round(x.numel() ** 0.5))
    if n * n != x.numel() or y.numel() != x.numel():
        raise ValueError("x and y must hold n x n values")
    if method not in ("pearson", "spearman"):
        raise ValueError("method must be 'pearson' or 'spearman'")
    perms = (np.ascontiguousarray(perms, dtype=np.int32).reshape(-1, n) if n > 0
             else np.zeros((0, 0), np.int32))
    m = perms.shape[0]
    stats = np.zeros(m, np.float64)
    r, p = ctypes.c_double(), ctypes.c_double()
    precision = FP64 if x.dtype == torch.float64 else MIXED
    status = load().unifrac_mantel(
        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), precision, n,
        perms.ctypes.data_as(ctypes.c_void_p) if m else None, m,
        MANTEL_SPEARMAN if method == "spearman" else MANTEL_PEARSON,
        ctypes.byref(r), stats.ctypes.data_as(ctypes.c_void_p), ctypes.byref(p),
        _stream_handle(stream))
    _check(status)
    return float(r.value), stats, float(p.value)


def unifrac_check_bounded_wait(limit_us: int, stream=None) -> int:
    """Runs the device-side bounded wait on an mbarrier that nothing
    completes; returns the status the kernel recorded (UNIFRAC_E_DEVICE_TIMEOUT
    = -8 when the bound works)."""
    status = ctypes.c_int32(0)
    _check(load().unifrac_check_bounded_wait(int(limit_us), ctypes.byref(status),
                                             _stream_handle(stream)))
    return int(status.value)


def unifrac_measure_peak(pipe: int, stream=None) -> float:
    """Measured FMA instructions per second of one pipe (PEAK_FP32_FMA or
    PEAK_FP64_FMA) of the current device."""
    v = ctypes.c_double()
    _check(load().unifrac_measure_peak(int(pipe), ctypes.byref(v), _stream_handle(stream)))
    return float(v.value)


def unifrac_set_memory_cache(max_bytes: int, device: int = -1) -> None:
    """Most bytes the library's cache of device blocks may hold on a device
    (-1: the current one); 0 turns it off, -1 restores the default (half the
    device's memory)."""
    _check(load().unifrac_set_memory_cache(int(device), int(max_bytes)))


def unifrac_release_cached_memory(device: int = -1) -> None:
    """Frees every block the cache holds on a device (-1: on every device)."""
    _check(load().unifrac_release_cached_memory(int(device)))


def unifrac_cached_memory(device: int = -1) -> int:
    """Bytes the cache holds on a device (-1: the current one)."""
    v = ctypes.c_int64()
    _check(load().unifrac_cached_memory(int(device), ctypes.byref(v)))
    return int(v.value)


def unifrac_destroy(ctx) -> None:
    if ctx:
        load().unifrac_destroy(ctx)


def unifrac_set_option(ctx, option: int, value: int) -> None:
    _check(load().unifrac_set_option(ctx, option, int(value)), ctx)


def unifrac_get_option(ctx, option: int) -> int:
    v = ctypes.c_int64()
    _check(load().unifrac_get_option(ctx, option, ctypes.byref(v)), ctx)
    return int(v.value)


def unifrac_autotune(ctx, variant: int, precision: int, out, repeats: int = 2) -> None:
    """Times the kernel settings of one (variant, precision) on the device
    and keeps the fastest as the context's options; `out` is a device buffer
    of at least unifrac_output_bytes(ctx, precision, OUT_CONDENSED) bytes,
    overwritten."""
    ptr, nbytes = _data_ptr(out)
    _check(load().unifrac_autotune(ctx, int(variant), int(precision), ctypes.c_void_p(ptr),
                                   nbytes, int(repeats)), ctx)


def unifrac_get_stat(ctx, stat: int) -> float:
    v = ctypes.c_double()
    _check(load().unifrac_get_stat(ctx, stat, ctypes.byref(v)), ctx)
    return float(v.value)


class Context:
    """Owning wrapper around a context (closes on exit / garbage collection)."""

    def __init__(self, tree, table, stream=None):
        self.n_samples = table.n_samples
        self.study_offsets = table.study_offsets
        self.handle = unifrac_create(tree.parent, tree.length, table.feature_node,
                                     table.indptr, table.indices, table.counts,
                                     table.n_samples, table.study_offsets, stream)

    def close(self) -> None:
        if getattr(self, "handle", None):
            unifrac_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def output_bytes(self, precision, layout, stripe_start=0, stripe_stop=-1) -> int:
        return unifrac_output_bytes(self.handle, precision, layout, stripe_start, stripe_stop)

    def run(self, variant, precision, layout=OUT_FULL, stripe_start=0, stripe_stop=-1,
            out=None, device="cuda"):
        """Run and return `out` (allocated as a torch tensor on `device` if None)."""
        if out is None:
            import torch
            nbytes = self.output_bytes(precision, layout, stripe_start, stripe_stop)
            if variant == BOTH:
                nbytes *= 2
            dt = torch.float64 if precision == FP64 else torch.float32
            out = torch.zeros(nbytes // (8 if precision == FP64 else 4), dtype=dt, device=device)
        unifrac_run(self.handle, variant, precision, stripe_start, stripe_stop, layout, out)
        return out

    def run_streamed(self, variant, precision, layout, chunk_stripes, out=None):
        """Host matrix computed in chunks of stripes (numpy array returned)."""
        if out is None:
            nbytes = self.output_bytes(precision, layout) * (2 if variant == BOTH else 1)
            out = np.empty(nbytes // (8 if precision == FP64 else 4),
                           np.float64 if precision == FP64 else np.float32)
        unifrac_run_streamed(self.handle, variant, precision, layout, out, chunk_stripes)
        return out

    def set_option(self, option, value) -> None:
        unifrac_set_option(self.handle, option, value)

    def get_option(self, option) -> int:
        return unifrac_get_option(self.handle, option)

    def stat(self, stat) -> float:
        return unifrac_get_stat(self.handle, stat)

    def n_stripes(self, study: int = 0) -> int:
        return unifrac_n_stripes(self.handle, study)
