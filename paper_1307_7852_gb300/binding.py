"""ctypes binding of libknng.so (the C ABI declared in include/knng.h).

Argument marshalling only: tensors become device pointers, the current torch
stream becomes the cudaStream_t, and every step of the computation runs in
the library's CUDA kernels.  There is no fallback: if the shared library is
missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libknng.so")

KNNG_OK = 0
DTYPE_F32, DTYPE_F16, DTYPE_U8 = 0, 1, 2
PREC_FP32, PREC_BF16, PREC_FP8E4M3 = 0, 1, 2
PART_RANDOM, PART_PCA, PART_FEATURES, PART_FEATURES_PCA = 0, 1, 2, 3
METRIC_L2, METRIC_COSINE = 0, 1
PROP_FIRST_ORDER, PROP_BEST_FIRST, PROP_PAIRWISE = 0, 1, 2

_lock = threading.Lock()
_lib = None
_handles = {}


class KnngError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"knng error {code}: {msg}")
        self.code = code


class knng_dataset(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("d", ctypes.c_int32),
                ("n", ctypes.c_int64), ("ld", ctypes.c_int64), ("ids", ctypes.c_void_p),
                ("dists", ctypes.c_void_p)]


class knng_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("T", ctypes.c_int32), ("leaf_size", ctypes.c_int32),
                ("prop_rounds", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("rescore_mult", ctypes.c_int32),
                ("partitioner", ctypes.c_int32), ("metric", ctypes.c_int32),
                ("propagation", ctypes.c_int32), ("budget", ctypes.c_int32), ("r_stop", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


# exported entry points -> argtypes
_P, _I32, _I64, _U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
SIGNATURES = {
    "knng_create": [ctypes.POINTER(ctypes.c_void_p), _I32],
    "knng_destroy": [_P],
    "knng_status_string": [_I32],
    "knng_last_error": [_P],
    "knng_leaf_count": [_I64, _I32, ctypes.POINTER(ctypes.c_int64)],
    "knng_leaf_offsets": [_I64, _I32, _P],
    "knng_build": [_P, _P, _I32, _I64, _I32, _I64, ctypes.POINTER(knng_params), _P, _P, _P],
    "knng_build_host": [_P, _P, _I32, _I64, _I32, _I64, ctypes.POINTER(knng_params), _P, _P, _P],
    "knng_partition": [_P, _P, _I32, _I64, _I32, _I64, _I32, _I32, _U64, _P, _P],
    "knng_leaf_knn": [_P, _P, _I32, _I64, _I32, _I64, _I32, _I32, _P, _I32, _I32, _I32, _P, _P, _P],
    "knng_merge": [_P, _I64, _I32, _I32, _P, _P, _P, _P, _P],
    "knng_propagate": [_P, _P, _I32, _I64, _I32, _I64, _I32, _I32, _P, _P, _P, _P, _P],
    "knng_propagate_best_first": [_P, _P, _I32, _I64, _I32, _I64, _I32, _I32, _I32, _P, _P, _P, _P],
    "knng_propagate_pairwise": [_P, _P, _I32, _I64, _I32, _I64, _I32, _I32, _P, _P, _P, _P, _P],
    "knng_divisions_used": [_P, _P, _P, _I32],
    "knng_split_levels": [_I64, _I32, _P],
    "knng_partition_pca": [_P, _P, _I32, _I64, _I32, _I64, _I32, _I32, _U64, _P, _P, _P],
    "knng_normalize_rows": [_P, _P, _I32, _I64, _I32, _I64, _P, _I64, _P],
    "knng_exact_knn": [_P, _P, _I32, _I64, _I32, _I64, _P, _I64, _I32, _P, _P, _P],
    "knng_set_stage_events": [_P, _P, _I32],
    "knng_launch_counter": [ctypes.POINTER(ctypes.c_uint64)],
    "knng_sync": [_P, _P],
    "knng_set_wait_limit": [_P, _I64],
    "knng_set_propagation_counters": [_P, _P, _I32],
    "knng_autotune": [_P, _P, _I32, _I64, _I32, _I64, ctypes.POINTER(knng_params), _P, _P, _P, _P],
    "knng_tune_save": [_P, ctypes.c_char_p],
    "knng_tune_load": [_P, ctypes.c_char_p],
    "knng_mlp_create": [_I32, _I32, _I32, _I32, _U64, ctypes.POINTER(ctypes.c_void_p)],
    "knng_mlp_destroy": [_P],
    "knng_mlp_param_count": [_P, ctypes.POINTER(ctypes.c_int64)],
    "knng_mlp_get_params": [_P, _P],
    "knng_mlp_set_params": [_P, _P],
    "knng_mlp_get_adam_state": [_P, _P, _P, ctypes.POINTER(ctypes.c_int64)],
    "knng_mlp_set_adam_state": [_P, _P, _P, _I64],
    "knng_mlp_loss_grad": [_P, _P, _I32, ctypes.POINTER(ctypes.c_float), _P, _P],
    "knng_mlp_train": [_P, _P, _I32, _I64, _I32, _I64, _P, _I32, _I32, _I32, ctypes.c_float, _U64,
                       ctypes.POINTER(ctypes.c_float), _P],
    "knng_mlp_save": [_P, ctypes.c_char_p],
    "knng_mlp_load": [_P, ctypes.c_char_p],
    "knng_mlp_forward": [_P, _P, _P, _I32, _I64, _I32, _I64, _P, _P],
    "knng_build_learned": [_P, _P, _P, _I32, _I64, _I32, _I64, ctypes.POINTER(knng_params), _P, _P, _P],
    "knng_partition_learned": [_P, _P, _P, _I32, _I64, _I32, _I64, _I32, _I32, _U64, _P, _P, _P],
    "knng_build_batched": [_P, _I32, _P, ctypes.POINTER(knng_params), _P],
    "knng_propagate_noalloc": [_P, _I32, _I64, _I32, _I64, _I32, _I32, _P, _P, _P, _P, _P],
}


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it was not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                                   "(the k-NN graph path has no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, argt in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = argt
                fn.restype = ctypes.c_int
            L.knng_status_string.restype = ctypes.c_char_p
            L.knng_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


class Handle:
    """Owns a knng_handle (device workspace + cached tree plan)."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        h = ctypes.c_void_p()
        rc = lib().knng_create(ctypes.byref(h), self.device)
        if rc != KNNG_OK:
            raise KnngError(rc, lib().knng_status_string(rc).decode())
        self._h = h

    @property
    def ptr(self):
        return self._h

    def check(self, rc: int, what: str):
        if rc != KNNG_OK:
            detail = lib().knng_last_error(self._h).decode()
            raise KnngError(rc, f"{what}: {lib().knng_status_string(rc).decode()}: {detail}")

    def close(self):
        if getattr(self, "_h", None):
            lib().knng_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def handle(device: int = 0) -> Handle:
    """A per-device handle shared by the convenience calls below."""
    with _lock:
        h = _handles.get(device)
    if h is None:
        h = Handle(device)
        with _lock:
            _handles[device] = h
    return h


# ------------------------------------------------------------ marshalling --
def _torch():
    import torch
    return torch


def _xdesc(X):
    torch = _torch()
    if not isinstance(X, torch.Tensor) or not X.is_cuda:
        raise TypeError("X must be a CUDA tensor")
    if X.dim() != 2 or X.stride(1) != 1:
        raise ValueError("X must be 2-D with unit stride along d")
    if X.dtype == torch.float32:
        dt = DTYPE_F32
    elif X.dtype == torch.float16:
        dt = DTYPE_F16
    elif X.dtype == torch.uint8:
        dt = DTYPE_U8
    else:
        raise TypeError("X must be float32, float16 or uint8")
    return ctypes.c_void_p(X.data_ptr()), dt, X.shape[0], X.shape[1], X.stride(0)


def _stream(dev, stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _out(shape, dtype, device, given):
    torch = _torch()
    if given is not None:
        if tuple(given.shape) != tuple(shape) or given.dtype != dtype or not given.is_contiguous():
            raise ValueError(f"output must be contiguous {dtype} {tuple(shape)}")
        return given
    return torch.empty(shape, dtype=dtype, device=device)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def make_params(k, T, leaf_size, prop_rounds, seed, precision=PREC_FP32, rescore_mult=2,
                partitioner=PART_RANDOM, metric=0, propagation=0, budget=0, r_stop=0.0) -> knng_params:
    return knng_params(int(k), int(T), int(leaf_size), int(prop_rounds), int(seed) & (2**64 - 1),
                       int(precision), int(rescore_mult), int(partitioner), int(metric), int(propagation),
                       int(budget), float(r_stop), 0)


# ----------------------------------------------------------- entry points --
def knng_leaf_count(n: int, leaf_size: int) -> int:
    out = ctypes.c_int64()
    rc = lib().knng_leaf_count(int(n), int(leaf_size), ctypes.byref(out))
    if rc != KNNG_OK:
        raise KnngError(rc, "knng_leaf_count")
    return int(out.value)


def knng_leaf_offsets(n: int, leaf_size: int) -> np.ndarray:
    off = np.zeros(knng_leaf_count(n, leaf_size) + 1, dtype=np.int64)
    rc = lib().knng_leaf_offsets(int(n), int(leaf_size), ctypes.c_void_p(off.ctypes.data))
    if rc != KNNG_OK:
        raise KnngError(rc, "knng_leaf_offsets")
    return off


def knng_build(X, k, T, leaf_size, prop_rounds, seed, precision=PREC_FP32, rescore_mult=2,
               ids=None, dists=None, stream=None, h: Handle = None, metric: int = METRIC_L2,
               propagation: int = PROP_FIRST_ORDER, budget: int = 0, r_stop: float = 0.0,
               partitioner: int = PART_RANDOM):
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    h = h or handle(X.device.index or 0)
    ids = _out((n, k), torch.int32, X.device, ids)
    dists = _out((n, k), torch.float32, X.device, dists)
    p = make_params(k, T, leaf_size, prop_rounds, seed, precision, rescore_mult, metric=metric,
                    propagation=propagation, budget=budget, r_stop=r_stop, partitioner=partitioner)
    h.check(lib().knng_build(h.ptr, xp, dt, n, d, ld, ctypes.byref(p), _ptr(ids), _ptr(dists),
                             _stream(X.device, stream)), "knng_build")
    return ids, dists


def knng_build_host(X: np.ndarray, k, T, leaf_size, prop_rounds, seed, precision=PREC_FP32,
                    rescore_mult=2, ids=None, dists=None, stream=None, device: int = 0,
                    h: Handle = None, metric: int = METRIC_L2, propagation: int = PROP_FIRST_ORDER,
                    budget: int = 0, r_stop: float = 0.0, partitioner: int = PART_RANDOM):
    """Host arrays in and out (X float32/float16/uint8 [n, d], unit stride along d)."""
    X = np.asarray(X)
    if X.ndim != 2 or X.strides[1] != X.itemsize:
        raise ValueError("X must be 2-D with unit stride along d")
    dts = {np.dtype(np.float32): DTYPE_F32, np.dtype(np.float16): DTYPE_F16, np.dtype(np.uint8): DTYPE_U8}
    if X.dtype not in dts:
        raise TypeError("X must be float32, float16 or uint8")
    dt = dts[X.dtype]
    n, d = X.shape
    ld = X.strides[0] // X.itemsize
    if ids is None:
        ids = np.empty((n, k), dtype=np.int32)
    if dists is None:
        dists = np.empty((n, k), dtype=np.float32)
    h = h or handle(device)
    p = make_params(k, T, leaf_size, prop_rounds, seed, precision, rescore_mult, metric=metric,
                    propagation=propagation, budget=budget, r_stop=r_stop, partitioner=partitioner)
    torch = _torch()
    st = _stream(torch.device("cuda", device), stream)
    h.check(lib().knng_build_host(h.ptr, ctypes.c_void_p(X.ctypes.data), dt, n, d, ld, ctypes.byref(p),
                                  ctypes.c_void_p(ids.ctypes.data), ctypes.c_void_p(dists.ctypes.data), st),
            "knng_build_host")
    return ids, dists


def knng_partition(X, T, leaf_size, seed, perm=None, stream=None, h: Handle = None):
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    h = h or handle(X.device.index or 0)
    perm = _out((T, n), torch.int32, X.device, perm)
    h.check(lib().knng_partition(h.ptr, xp, dt, n, d, ld, int(T), int(leaf_size), int(seed) & (2**64 - 1),
                                 _ptr(perm), _stream(X.device, stream)), "knng_partition")
    return perm


def knng_split_levels(n: int, leaf_size: int) -> int:
    out = ctypes.c_int32()
    rc = lib().knng_split_levels(int(n), int(leaf_size), ctypes.byref(out))
    if rc != KNNG_OK:
        raise KnngError(rc, "knng_split_levels")
    return int(out.value)


def knng_partition_pca(X, T, leaf_size, seed, perm=None, with_dirs=False, stream=None, h: Handle = None):
    """Principal-direction trees; returns perm [T, n] (and, with with_dirs,
    the directions [T, 2^L - 1, d] by (level, node))."""
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    h = h or handle(X.device.index or 0)
    perm = _out((T, n), torch.int32, X.device, perm)
    dirs = None
    if with_dirs:
        L = knng_split_levels(n, leaf_size)
        dirs = torch.zeros((T, 2 ** L - 1, d), dtype=torch.float32, device=X.device)
    h.check(lib().knng_partition_pca(h.ptr, xp, dt, n, d, ld, int(T), int(leaf_size), int(seed) & (2**64 - 1),
                                     _ptr(perm), _ptr(dirs) if dirs is not None else None,
                                     _stream(X.device, stream)), "knng_partition_pca")
    return (perm, dirs) if with_dirs else perm


def knng_leaf_knn(X, T, leaf_size, perm, k, precision=PREC_FP32, rescore_mult=2, ids=None,
                  dists=None, stream=None, h: Handle = None):
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    h = h or handle(X.device.index or 0)
    if perm.dtype != torch.int32 or tuple(perm.shape) != (T, n) or not perm.is_contiguous():
        raise ValueError("perm must be contiguous int32 [T, n]")
    ids = _out((T, n, k), torch.int32, X.device, ids)
    dists = _out((T, n, k), torch.float32, X.device, dists)
    h.check(lib().knng_leaf_knn(h.ptr, xp, dt, n, d, ld, int(T), int(leaf_size), _ptr(perm), int(k),
                                int(precision), int(rescore_mult), _ptr(ids), _ptr(dists),
                                _stream(X.device, stream)), "knng_leaf_knn")
    return ids, dists


def knng_merge(ids_in, dists_in, ids=None, dists=None, stream=None, h: Handle = None):
    torch = _torch()
    T, n, k = ids_in.shape
    for t_, dt_ in ((ids_in, torch.int32), (dists_in, torch.float32)):
        if t_.dtype != dt_ or not t_.is_contiguous() or not t_.is_cuda or tuple(t_.shape) != (T, n, k):
            raise ValueError("inputs must be contiguous CUDA [T, n, k] int32 / float32")
    h = h or handle(ids_in.device.index or 0)
    ids = _out((n, k), torch.int32, ids_in.device, ids)
    dists = _out((n, k), torch.float32, ids_in.device, dists)
    h.check(lib().knng_merge(h.ptr, n, T, k, _ptr(ids_in), _ptr(dists_in), _ptr(ids), _ptr(dists),
                             _stream(ids_in.device, stream)), "knng_merge")
    return ids, dists


def knng_propagate(X, ids_in, dists_in, rounds=1, ids=None, dists=None, stream=None, h: Handle = None):
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    k = ids_in.shape[1]
    for t_, dt_ in ((ids_in, torch.int32), (dists_in, torch.float32)):
        if t_.dtype != dt_ or not t_.is_contiguous() or tuple(t_.shape) != (n, k):
            raise ValueError("inputs must be contiguous [n, k] int32 / float32")
    h = h or handle(X.device.index or 0)
    ids = _out((n, k), torch.int32, X.device, ids)
    dists = _out((n, k), torch.float32, X.device, dists)
    h.check(lib().knng_propagate(h.ptr, xp, dt, n, d, ld, int(k), int(rounds), _ptr(ids_in),
                                 _ptr(dists_in), _ptr(ids), _ptr(dists), _stream(X.device, stream)),
            "knng_propagate")
    return ids, dists


def knng_propagate_best_first(X, ids_in, budget, rounds=1, ids=None, dists=None, stream=None, h: Handle = None):
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    k = ids_in.shape[1]
    h = h or handle(X.device.index or 0)
    ids = _out((n, k), torch.int32, X.device, ids)
    dists = _out((n, k), torch.float32, X.device, dists)
    h.check(lib().knng_propagate_best_first(h.ptr, xp, dt, n, d, ld, k, int(budget), int(rounds), _ptr(ids_in),
                                            _ptr(ids), _ptr(dists), _stream(X.device, stream)),
            "knng_propagate_best_first")
    return ids, dists


def knng_propagate_pairwise(X, ids_in, dists_in, rounds=1, ids=None, dists=None, stream=None, h: Handle = None):
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    k = ids_in.shape[1]
    h = h or handle(X.device.index or 0)
    ids = _out((n, k), torch.int32, X.device, ids)
    dists = _out((n, k), torch.float32, X.device, dists)
    h.check(lib().knng_propagate_pairwise(h.ptr, xp, dt, n, d, ld, k, int(rounds), _ptr(ids_in), _ptr(dists_in),
                                          _ptr(ids), _ptr(dists), _stream(X.device, stream)),
            "knng_propagate_pairwise")
    return ids, dists


def knng_divisions_used(h: Handle = None, device: int = 0, cap: int = 32):
    """(divisions used by the last build on h, their effective rates)."""
    h = h or handle(device)
    m = ctypes.c_int32()
    rates = (ctypes.c_float * cap)()
    rc = lib().knng_divisions_used(h.ptr, ctypes.byref(m), rates, cap)
    if rc != KNNG_OK:
        raise KnngError(rc, "knng_divisions_used")
    return int(m.value), [float(r) for r in rates[:min(cap, m.value)]]


def knng_normalize_rows(X, out=None, stream=None, h: Handle = None):
    """Rows of X (CUDA tensor) scaled to unit length in FP32 (cosine metric)."""
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    h = h or handle(X.device.index or 0)
    out = _out((n, d), torch.float32, X.device, out)
    h.check(lib().knng_normalize_rows(h.ptr, xp, dt, n, d, ld, _ptr(out), d, _stream(X.device, stream)),
            "knng_normalize_rows")
    return out


def knng_exact_knn(X, queries, k, ids=None, dists=None, stream=None, h: Handle = None):
    """Exact k-NN lists of the query ids (device int32 [nq]) against all points."""
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    if queries.dtype != torch.int32 or not queries.is_contiguous() or not queries.is_cuda:
        raise ValueError("queries must be a contiguous CUDA int32 tensor")
    nq = queries.shape[0]
    h = h or handle(X.device.index or 0)
    ids = _out((nq, k), torch.int32, X.device, ids)
    dists = _out((nq, k), torch.float32, X.device, dists)
    h.check(lib().knng_exact_knn(h.ptr, xp, dt, n, d, ld, _ptr(queries), nq, int(k), _ptr(ids),
                                 _ptr(dists), _stream(X.device, stream)), "knng_exact_knn")
    return ids, dists


def knng_set_stage_events(events, h: Handle):
    """Record the given torch.cuda.Event objects at the stage boundaries of
    knng_build on handle h (events=None stops recording)."""
    if not events:
        h.check(lib().knng_set_stage_events(h.ptr, None, 0), "knng_set_stage_events")
        return
    arr = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
    h.check(lib().knng_set_stage_events(h.ptr, arr, len(events)), "knng_set_stage_events")


def knng_set_wait_limit(cycles: int, h: Handle):
    """Limit (SM cycles, 0 = about one second) of the tensor-core leaf
    kernel's pipeline waits for later calls on h."""
    h.check(lib().knng_set_wait_limit(h.ptr, int(cycles)), "knng_set_wait_limit")


def knng_set_propagation_counters(counters, h: Handle):
    """counters: CUDA int64 tensor of 2 * rounds zeros (rows scored, list
    slots loaded per first-order round of later calls on h), or None."""
    if counters is None:
        h.check(lib().knng_set_propagation_counters(h.ptr, None, 0), "knng_set_propagation_counters")
        return
    assert counters.numel() % 2 == 0
    h.check(lib().knng_set_propagation_counters(h.ptr, _ptr(counters), int(counters.numel() // 2)),
            "knng_set_propagation_counters")


def knng_launch_counter() -> int:
    """Kernels launched by the library in this process so far."""
    out = ctypes.c_uint64()
    rc = lib().knng_launch_counter(ctypes.byref(out))
    if rc != KNNG_OK:
        raise KnngError(rc, "knng_launch_counter")
    return int(out.value)


def knng_sync(h: Handle = None, stream=None, device: int = 0):
    """Synchronise the stream and raise if a bounded device wait gave up."""
    torch = _torch()
    h = h or handle(device)
    h.check(lib().knng_sync(h.ptr, _stream(torch.device("cuda", h.device), stream)), "knng_sync")


def knng_propagate_noalloc(X, ids_in, dists_in, rounds=1, ids=None, dists=None, stream=None):
    """Propagation rounds that allocate no device memory (for callers that
    cannot allocate on their call path); the lists between rounds live in the
    library's fixed 16 MiB device array.  Runs on X's device, which is made
    current.  Outputs, if given, must be preallocated by the caller."""
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    k = ids_in.shape[1]
    ids = _out((n, k), torch.int32, X.device, ids)
    dists = _out((n, k), torch.float32, X.device, dists)
    with torch.cuda.device(X.device):
        rc = lib().knng_propagate_noalloc(xp, dt, n, d, ld, int(k), int(rounds), _ptr(ids_in), _ptr(dists_in),
                                          _ptr(ids), _ptr(dists), _stream(X.device, stream))
    if rc != KNNG_OK:
        raise KnngError(rc, "knng_propagate_noalloc: " + lib().knng_status_string(rc).decode())
    return ids, dists


def knng_build_batched(Xs, k, T, leaf_size, prop_rounds, seed, precision=PREC_FP32, rescore_mult=2,
                       outs=None, stream=None, h: Handle = None, metric: int = METRIC_L2,
                       propagation: int = PROP_FIRST_ORDER, budget: int = 0, r_stop: float = 0.0):
    """Graphs of many independent point sets (CUDA tensors) in one recorded
    launch; returns a list of (ids, dists) per set."""
    torch = _torch()
    if not Xs:
        raise ValueError("no point sets")
    dev = Xs[0].device
    h = h or handle(dev.index or 0)
    arr = (knng_dataset * len(Xs))()
    res = []
    for i, X in enumerate(Xs):
        xp, dt, n, d, ld = _xdesc(X)
        oi, od = (outs[i] if outs is not None else (None, None))
        oi = _out((n, k), torch.int32, dev, oi)
        od = _out((n, k), torch.float32, dev, od)
        arr[i] = knng_dataset(xp.value, dt, d, n, ld, oi.data_ptr(), od.data_ptr())
        res.append((oi, od))
    p = make_params(k, T, leaf_size, prop_rounds, seed, precision, rescore_mult, metric=metric,
                    propagation=propagation, budget=budget, r_stop=r_stop)
    h.check(lib().knng_build_batched(h.ptr, len(Xs), arr, ctypes.byref(p), _stream(dev, stream)),
            "knng_build_batched")
    return res


def knng_autotune(X, k, T, leaf_size, seed, precision=PREC_BF16, rescore_mult=2, prop_rounds=0,
                  stream=None, h: Handle = None):
    """Tunes the tensor-core leaf tiles for X's shape on handle h; returns
    (stages, rows_per_group, ms)."""
    xp, dt, n, d, ld = _xdesc(X)
    h = h or handle(X.device.index or 0)
    p = make_params(k, T, leaf_size, prop_rounds, seed, precision, rescore_mult)
    S, RG, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    h.check(lib().knng_autotune(h.ptr, xp, dt, n, d, ld, ctypes.byref(p), ctypes.byref(S), ctypes.byref(RG),
                                ctypes.byref(ms), _stream(X.device, stream)), "knng_autotune")
    return S.value, RG.value, ms.value


def knng_tune_save(path: str, h: Handle):
    h.check(lib().knng_tune_save(h.ptr, os.fsencode(path)), "knng_tune_save")


def knng_tune_load(path: str, h: Handle):
    h.check(lib().knng_tune_load(h.ptr, os.fsencode(path)), "knng_tune_load")


class Mlp:
    """The learned partitioner's split-feature network (knng_mlp)."""

    def __init__(self, d_in, hidden=256, d_out=16, seed=0, device=0):
        p = ctypes.c_void_p()
        rc = lib().knng_mlp_create(int(device), int(d_in), int(hidden), int(d_out), int(seed), ctypes.byref(p))
        if rc != KNNG_OK:
            raise KnngError(rc, "knng_mlp_create: " + lib().knng_status_string(rc).decode())
        self._p, self.d_in, self.hidden, self.d_out, self.device = p, d_in, hidden, d_out, device

    @property
    def ptr(self):
        return self._p

    def _chk(self, rc, what):
        if rc != KNNG_OK:
            raise KnngError(rc, what + ": " + lib().knng_status_string(rc).decode())

    def param_count(self) -> int:
        c = ctypes.c_int64()
        self._chk(lib().knng_mlp_param_count(self._p, ctypes.byref(c)), "knng_mlp_param_count")
        return int(c.value)

    def get_params(self):
        """(W1, b1, W2, b2) as float32 numpy arrays."""
        buf = np.empty(self.param_count(), dtype=np.float32)
        self._chk(lib().knng_mlp_get_params(self._p, ctypes.c_void_p(buf.ctypes.data)), "knng_mlp_get_params")
        H, d, C = self.hidden, self.d_in, self.d_out
        o = 0
        W1 = buf[o:o + H * d].reshape(H, d); o += H * d
        b1 = buf[o:o + H]; o += H
        W2 = buf[o:o + C * H].reshape(C, H); o += C * H
        b2 = buf[o:o + C]
        return W1, b1, W2, b2

    def set_params(self, W1, b1, W2, b2):
        buf = np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2)]).astype(np.float32)
        assert buf.size == self.param_count()
        self._chk(lib().knng_mlp_set_params(self._p, ctypes.c_void_p(buf.ctypes.data)), "knng_mlp_set_params")

    def get_adam_state(self):
        """(m1, m2, t): Adam moment estimates (float32 numpy) and steps taken."""
        m1 = np.empty(self.param_count(), dtype=np.float32)
        m2 = np.empty_like(m1)
        t = ctypes.c_int64()
        self._chk(lib().knng_mlp_get_adam_state(self._p, ctypes.c_void_p(m1.ctypes.data),
                                                ctypes.c_void_p(m2.ctypes.data), ctypes.byref(t)),
                  "knng_mlp_get_adam_state")
        return m1, m2, int(t.value)

    def set_adam_state(self, m1, m2, t):
        m1 = np.ascontiguousarray(m1, dtype=np.float32)
        m2 = np.ascontiguousarray(m2, dtype=np.float32)
        assert m1.size == m2.size == self.param_count()
        self._chk(lib().knng_mlp_set_adam_state(self._p, ctypes.c_void_p(m1.ctypes.data),
                                                ctypes.c_void_p(m2.ctypes.data), int(t)),
                  "knng_mlp_set_adam_state")

    def loss_grad(self, Xpairs, stream=None):
        """Loss and packed gradient of a batch (CUDA float32 [2B, d_in])."""
        torch = _torch()
        B = Xpairs.shape[0] // 2
        g = torch.empty(self.param_count(), dtype=torch.float32, device=Xpairs.device)
        loss = ctypes.c_float()
        self._chk(lib().knng_mlp_loss_grad(self._p, _ptr(Xpairs), int(B), ctypes.byref(loss), _ptr(g),
                                           _stream(Xpairs.device, stream)), "knng_mlp_loss_grad")
        return float(loss.value), g

    def train(self, X, ids, steps, batch_edges=4096, lr=1e-3, seed=0, stream=None) -> float:
        xp, dt, n, d, ld = _xdesc(X)
        k = ids.shape[1]
        loss = ctypes.c_float()
        self._chk(lib().knng_mlp_train(self._p, xp, dt, n, d, ld, _ptr(ids), int(k), int(steps), int(batch_edges),
                                       float(lr), int(seed), ctypes.byref(loss), _stream(X.device, stream)),
                  "knng_mlp_train")
        return float(loss.value)

    def save(self, path):
        self._chk(lib().knng_mlp_save(self._p, os.fsencode(path)), "knng_mlp_save")

    def load(self, path):
        self._chk(lib().knng_mlp_load(self._p, os.fsencode(path)), "knng_mlp_load")

    def close(self):
        if getattr(self, "_p", None):
            lib().knng_mlp_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def knng_mlp_forward(mlp: Mlp, X, Z=None, stream=None, h: Handle = None):
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    h = h or handle(X.device.index or 0)
    Z = _out((n, mlp.d_out), torch.float32, X.device, Z)
    h.check(lib().knng_mlp_forward(h.ptr, mlp.ptr, xp, dt, n, d, ld, _ptr(Z), _stream(X.device, stream)),
            "knng_mlp_forward")
    return Z


def knng_build_learned(mlp: Mlp, X, k, T, leaf_size, prop_rounds, seed, precision=PREC_FP32, rescore_mult=2,
                       ids=None, dists=None, stream=None, h: Handle = None, propagation: int = PROP_FIRST_ORDER,
                       budget: int = 0, r_stop: float = 0.0, partitioner: int = PART_RANDOM):
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    h = h or handle(X.device.index or 0)
    ids = _out((n, k), torch.int32, X.device, ids)
    dists = _out((n, k), torch.float32, X.device, dists)
    p = make_params(k, T, leaf_size, prop_rounds, seed, precision, rescore_mult, propagation=propagation,
                    budget=budget, r_stop=r_stop, partitioner=partitioner)
    h.check(lib().knng_build_learned(h.ptr, mlp.ptr, xp, dt, n, d, ld, ctypes.byref(p), _ptr(ids), _ptr(dists),
                                     _stream(X.device, stream)), "knng_build_learned")
    return ids, dists


def knng_partition_learned(mlp: Mlp, X, T, leaf_size, seed, perm=None, with_z=False, stream=None,
                           h: Handle = None):
    """Canonical leaf sets of the per-level learned-feature splits
    (knng_build_learned's KNNG_PART_FEATURES partition): perm [T, n], and the
    network outputs Z [n, d_out] used when with_z."""
    torch = _torch()
    xp, dt, n, d, ld = _xdesc(X)
    h = h or handle(X.device.index or 0)
    perm = _out((T, n), torch.int32, X.device, perm)
    Z = torch.empty((n, mlp.d_out), dtype=torch.float32, device=X.device) if with_z else None
    h.check(lib().knng_partition_learned(h.ptr, mlp.ptr, xp, dt, n, d, ld, int(T), int(leaf_size),
                                         int(seed) & (2**64 - 1), _ptr(perm), _ptr(Z) if Z is not None else None,
                                         _stream(X.device, stream)), "knng_partition_learned")
    return (perm, Z) if with_z else perm
