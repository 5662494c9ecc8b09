"""CPU oracle for the k-NN graph method of arXiv:1307.7852 (Wang et al.).

TEST INFRASTRUCTURE.  This package is the plain, slow reference that the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library in
``paper_1307_7852_gb300`` never does, and the two share no code.

The arithmetic lives in ``knng_oracle.c`` (plain C, FP64 distances, compiled
with ``-ffp-contract=off``); this module compiles it with gcc, loads it with
ctypes and composes the stages in the order of the paper:

* ``partition``   -- one random partition tree (Sec. 3.1; App. after Lemma 1)
* ``partition_features`` -- one tree of the learned partitioner's per-level
  feature splits (not in the paper)
* ``leaf_knn``    -- brute force inside every leaf (Sec. 3.1)
* ``merge``       -- union of the T base graphs, k nearest kept (Sec. 3.1)
* ``propagate``   -- one first-order propagation round (Sec. 3.2, Theorem 1)
* ``knn_exact``   -- exact k-NN lists by brute force (Def. 1; Sec. 4)
* ``build_graph`` -- the whole method: T trees, merge, R rounds

Inputs of dtype float16 are widened to float32 first (exact).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knng_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PREC_FP32, PREC_BF16, PREC_FP8E4M3 = 0, 1, 2
METRIC_L2, METRIC_COSINE = 0, 1
PROP_FIRST_ORDER, PROP_BEST_FIRST, PROP_PAIRWISE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile knng_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i64, i32, u32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64
            lib.orc_philox4x32_10.argtypes = [P, P, P]
            lib.orc_direction.argtypes = [u64, u32, u32, u32, i32, P]
            lib.orc_project.argtypes = [P, P, i32]
            lib.orc_project.restype = ctypes.c_float
            lib.orc_ord.argtypes = [ctypes.c_float]
            lib.orc_ord.restype = u32
            lib.orc_leaf_count.argtypes = [i64, i32]
            lib.orc_leaf_count.restype = i64
            lib.orc_partition.argtypes = [P, i64, i32, i64, u64, u32, i32, P, P]
            lib.orc_partition_dirs.argtypes = [P, i64, i32, i64, P, i32, P, P]
            lib.orc_feature_order.argtypes = [u64, u32, i32, P]
            lib.orc_partition_features.argtypes = [P, i64, i32, i64, P, i32, u64, u32, i32, ctypes.c_float, P, P]
            lib.orc_leaf_knn.argtypes = [P, i64, i32, i64, P, P, i64, i32, P, P]
            lib.orc_leaf_knn_quant.argtypes = [P, i64, i32, i64, P, P, P, i64, i32, i32, P, P]
            lib.orc_merge.argtypes = [P, i64, i32, i64, i32, i32, P, P, P]
            lib.orc_propagate.argtypes = [P, i64, i32, i64, i32, P, P, P]
            lib.orc_propagate_rows.argtypes = [P, i64, i32, i64, i32, P, P, i64, P, P]
            lib.orc_knn_exact.argtypes = [P, i64, i32, i64, i32, P, i64, P, P]
            lib.orc_pair_dist.argtypes = [P, i32, i64, P, P, i64, P]
            lib.orc_normalize_rows.argtypes = [P, i64, i32, i64, P]
            lib.orc_canon_dist32.argtypes = [P, P, i32]
            lib.orc_canon_dist32.restype = ctypes.c_float
            lib.orc_propagate_best_first.argtypes = [P, i64, i32, i64, i32, P, i32, P, P]
            lib.orc_propagate_pairwise.argtypes = [P, i64, i32, i64, i32, P, P, P]
            lib.orc_bf16_round.argtypes = [ctypes.c_float]
            lib.orc_bf16_round.restype = ctypes.c_float
            lib.orc_e4m3_round.argtypes = [ctypes.c_float]
            lib.orc_e4m3_round.restype = ctypes.c_float
            lib.orc_quantize_rows.argtypes = [P, i64, i32, i64, i32, P, P]
            lib.orc_num_threads.restype = i32
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _as_f32(X) -> np.ndarray:
    X = np.asarray(X)
    if X.dtype == np.float16:
        X = X.astype(np.float32)
    return np.ascontiguousarray(X, dtype=np.float32)


def num_threads() -> int:
    return int(_load().orc_num_threads())


# --------------------------------------------------------------------- RNG --
def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def direction(seed: int, t: int, level: int, node: int, d: int) -> np.ndarray:
    lib = _load()
    a = np.zeros(d, dtype=np.float32)
    lib.orc_direction(seed, t, level, node, d, _ptr(a))
    return a


def project(x, a) -> np.float32:
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    a = np.ascontiguousarray(a, dtype=np.float32)
    assert x.shape == a.shape
    return np.float32(lib.orc_project(_ptr(x), _ptr(a), x.shape[0]))


def ord32(f: float) -> int:
    return int(_load().orc_ord(float(np.float32(f))))


# --------------------------------------------------------------- partition --
def leaf_count(n: int, g: int) -> int:
    return int(_load().orc_leaf_count(n, g))


def partition(X, seed: int, t: int, g: int):
    """Canonical leaf set of tree t: (perm int32[n], leaf_off int64[L+1])."""
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    perm = np.zeros(n, dtype=np.int32)
    off = np.zeros(leaf_count(n, g) + 1, dtype=np.int64)
    lib.orc_partition(_ptr(X), n, d, d, seed, t, g, _ptr(perm), _ptr(off))
    return perm, off


def partition_with_dirs(X, dirs, g: int):
    """Tree whose node (level, v) splits along dirs[2^level - 1 + v]."""
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    dirs = np.ascontiguousarray(dirs, dtype=np.float32)
    assert dirs.ndim == 2 and dirs.shape[1] == d
    perm = np.zeros(n, dtype=np.int32)
    off = np.zeros(leaf_count(n, g) + 1, dtype=np.int64)
    lib.orc_partition_dirs(_ptr(X), n, d, d, _ptr(dirs), g, _ptr(perm), _ptr(off))
    return perm, off


LEARNED_TAU = 0.02


def feature_order(seed: int, t: int, C: int) -> np.ndarray:
    """Tree t's order of the C learned features (Philox Fisher-Yates)."""
    out = np.zeros(C, dtype=np.int32)
    _load().orc_feature_order(seed, t, C, _ptr(out))
    return out


def partition_features(X, Z, seed: int, t: int, g: int, tau: float = LEARNED_TAU):
    """Canonical leaf set of tree t under the learned partitioner's
    per-level feature splits (Z: float32 [n, C] network outputs); random
    directions where a feature is flat in a node and past level C."""
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    Z = np.ascontiguousarray(Z, dtype=np.float32)
    assert Z.shape[0] == n
    C = Z.shape[1]
    perm = np.zeros(n, dtype=np.int32)
    off = np.zeros(leaf_count(n, g) + 1, dtype=np.int64)
    rc = lib.orc_partition_features(_ptr(X), n, d, d, _ptr(Z), C, seed, t, g, float(tau), _ptr(perm), _ptr(off))
    assert rc == 0
    return perm, off


def split_nodes(n: int, g: int):
    """(level, v, first position, size) of every split node of the tree
    shape (floor/ceil halving), in level order."""
    out = []
    level = [(0, n)]
    lvl = 0
    while level:
        nxt = []
        for v, (off, m) in enumerate(level):
            if m is None:
                nxt += [(0, None), (0, None)]
                continue
            if m > g:
                out.append((lvl, v, off, m))
                nxt += [(off, m // 2), (off + m // 2, m - m // 2)]
            else:
                nxt += [(0, None), (0, None)]
        if not any(m is not None for _, m in nxt):
            break
        level = nxt
        lvl += 1
    return out


# -------------------------------------------------------------- leaf graph --
def leaf_knn(X, perm, leaf_off, k: int):
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    leaf_off = np.ascontiguousarray(leaf_off, dtype=np.int64)
    ids = np.empty((n, k), dtype=np.int32)
    dists = np.empty((n, k), dtype=np.float32)
    lib.orc_leaf_knn(_ptr(X), n, d, d, _ptr(perm), _ptr(leaf_off), leaf_off.shape[0] - 1, k,
                     _ptr(ids), _ptr(dists))
    return ids, dists


def quantize_rows(X, precision: int):
    """Dequantised FP64 rows and per-row scales of the candidate-stage input."""
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    Xq = np.empty((n, d), dtype=np.float64)
    sc = np.empty(n, dtype=np.float32)
    lib.orc_quantize_rows(_ptr(X), n, d, d, int(precision), _ptr(Xq), _ptr(sc))
    return Xq, sc


def leaf_knn_quant(X, perm, leaf_off, k: int, kprime: int, precision: int):
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    Xq, _ = quantize_rows(X, precision)
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    leaf_off = np.ascontiguousarray(leaf_off, dtype=np.int64)
    ids = np.empty((n, k), dtype=np.int32)
    dists = np.empty((n, k), dtype=np.float32)
    lib.orc_leaf_knn_quant(_ptr(X), n, d, d, _ptr(Xq), _ptr(perm), _ptr(leaf_off),
                           leaf_off.shape[0] - 1, k, kprime, _ptr(ids), _ptr(dists))
    return ids, dists


def bf16_round(x: float) -> np.float32:
    return np.float32(_load().orc_bf16_round(float(np.float32(x))))


def e4m3_round(x: float) -> np.float32:
    return np.float32(_load().orc_e4m3_round(float(np.float32(x))))


# ------------------------------------------------------ merge / propagate --
def merge(X, lists, k: int):
    """lists: int32 [T, n, k] ids (-1 empty) -> (ids, dists) [n, k]."""
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    lists = np.ascontiguousarray(lists, dtype=np.int32)
    T = lists.shape[0]
    assert lists.shape == (T, n, k)
    ids = np.empty((n, k), dtype=np.int32)
    dists = np.empty((n, k), dtype=np.float32)
    lib.orc_merge(_ptr(X), n, d, d, T, k, _ptr(lists), _ptr(ids), _ptr(dists))
    return ids, dists


def propagate(X, ids_in, k: int):
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    ids_in = np.ascontiguousarray(ids_in, dtype=np.int32)
    assert ids_in.shape == (n, k)
    ids = np.empty((n, k), dtype=np.int32)
    dists = np.empty((n, k), dtype=np.float32)
    lib.orc_propagate(_ptr(X), n, d, d, k, _ptr(ids_in), _ptr(ids), _ptr(dists))
    return ids, dists


def propagate_rows(X, ids_in, k: int, rows):
    """One first-order round for the given points only: [len(rows), k]."""
    X = _as_f32(X)
    n, d = X.shape
    ids_in = np.ascontiguousarray(ids_in, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    ids = np.empty((rows.shape[0], k), dtype=np.int32)
    dists = np.empty((rows.shape[0], k), dtype=np.float32)
    _load().orc_propagate_rows(_ptr(X), n, d, d, k, _ptr(ids_in), _ptr(rows), rows.shape[0], _ptr(ids), _ptr(dists))
    return ids, dists


def canon_dist32(x, y) -> np.float32:
    """Canonical FP32 squared distance (32-lane order, pairwise rounds)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    return np.float32(_load().orc_canon_dist32(_ptr(x), _ptr(y), x.shape[0]))


def propagate_best_first(X, ids_in, k: int, budget: int):
    """One synchronous pass of budgeted best-first propagation (Sec. 3.2)."""
    X = _as_f32(X)
    n, d = X.shape
    ids_in = np.ascontiguousarray(ids_in, dtype=np.int32)
    assert ids_in.shape == (n, k) and budget >= k
    ids = np.empty((n, k), dtype=np.int32)
    dists = np.empty((n, k), dtype=np.float32)
    rc = _load().orc_propagate_best_first(_ptr(X), n, d, d, k, _ptr(ids_in), int(budget), _ptr(ids), _ptr(dists))
    assert rc == 0
    return ids, dists


def propagate_pairwise(X, ids_in, k: int):
    """One first-order round with pairwise updating (Sec. 3.4)."""
    X = _as_f32(X)
    n, d = X.shape
    ids_in = np.ascontiguousarray(ids_in, dtype=np.int32)
    assert ids_in.shape == (n, k)
    ids = np.empty((n, k), dtype=np.int32)
    dists = np.empty((n, k), dtype=np.float32)
    _load().orc_propagate_pairwise(_ptr(X), n, d, d, k, _ptr(ids_in), _ptr(ids), _ptr(dists))
    return ids, dists


def effective_rate(prev_ids, ids) -> float:
    """r_m of Sec. 3.2: the share of list entries after division m that were
    not in the lists after division m - 1 (padding -1 excluded)."""
    ids = np.asarray(ids)
    total = int(np.sum(ids >= 0))
    if prev_ids is None:
        return 1.0 if total else 0.0
    prev = np.asarray(prev_ids)
    new = 0
    for r in range(ids.shape[0]):
        cur = ids[r][ids[r] >= 0]
        new += int(np.sum(~np.isin(cur, prev[r])))
    return new / total if total else 0.0


def knn_exact(X, k: int, queries=None):
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    q = np.arange(n, dtype=np.int32) if queries is None else np.ascontiguousarray(queries, dtype=np.int32)
    ids = np.empty((q.shape[0], k), dtype=np.int32)
    dists = np.empty((q.shape[0], k), dtype=np.float32)
    lib.orc_knn_exact(_ptr(X), n, d, d, k, _ptr(q), q.shape[0], _ptr(ids), _ptr(dists))
    return ids, dists


def pair_dist(X, a, b) -> np.ndarray:
    lib = _load()
    X = _as_f32(X)
    n, d = X.shape
    a = np.ascontiguousarray(a, dtype=np.int32).ravel()
    b = np.ascontiguousarray(b, dtype=np.int32).ravel()
    out = np.empty(a.shape[0], dtype=np.float64)
    lib.orc_pair_dist(_ptr(X), d, d, _ptr(a), _ptr(b), a.shape[0], _ptr(out))
    return out


# ------------------------------------------------------------ whole method --
def normalize_rows(X) -> np.ndarray:
    """Rows scaled to unit length in FP32 (the cosine metric's input)."""
    X = _as_f32(X)
    n, d = X.shape
    out = np.empty((n, d), dtype=np.float32)
    _load().orc_normalize_rows(_ptr(X), n, d, X.strides[0] // 4, _ptr(out))
    return out


def build_graph(X, k: int, T: int, g: int, R: int, seed: int,
                precision: int = PREC_FP32, rescore_mult: int = 2, metric: int = METRIC_L2,
                r_stop: float = 0.0, prop: int = 0, budget: int = 0, info=None):
    """T random divisions, leaf graphs, merge, then R propagation rounds.

    metric = METRIC_COSINE: the same method on the rows scaled to unit length
    (normalize_rows), distances halved: 1 - cos of the scaled rows.
    r_stop > 0: divisions are added one by one until r_m < r_stop (at most
    T); info["divisions"] receives the number used, info["rates"] the r_m.
    prop: PROP_FIRST_ORDER (Theorem 1), PROP_BEST_FIRST (Sec. 3.2, visit
    budget `budget`) or PROP_PAIRWISE (first order with pairwise updating).
    """
    if metric == METRIC_COSINE:
        ids, dists = build_graph(normalize_rows(X), k, T, g, R, seed, precision, rescore_mult,
                                 r_stop=r_stop, prop=prop, budget=budget, info=info)
        return ids, (dists * np.float32(0.5)).astype(np.float32)
    X = _as_f32(X)
    n = X.shape[0]
    lists = np.empty((T, n, k), dtype=np.int32)
    ids = dists = None
    rates = []
    used = T
    for t in range(T):
        perm, off = partition(X, seed, t, g)
        if precision == PREC_FP32:
            lists[t], _ = leaf_knn(X, perm, off, k)
        else:
            lists[t], _ = leaf_knn_quant(X, perm, off, k, rescore_mult * k, precision)
        if r_stop > 0:
            # Sec. 4: add divisions until the m-th one's effective rate r_m
            # falls below the threshold, then start the propagation
            prev = ids
            ids, dists = merge(X, lists[:t + 1], k)
            rates.append(effective_rate(prev, ids))
            if rates[-1] < r_stop:
                used = t + 1
                break
    if r_stop <= 0:
        ids, dists = merge(X, lists, k)
    if info is not None:
        info["divisions"] = used
        info["rates"] = rates
    for _ in range(R):
        if prop == PROP_BEST_FIRST:
            ids, dists = propagate_best_first(X, ids, k, budget)
        elif prop == PROP_PAIRWISE:
            ids, dists = propagate_pairwise(X, ids, k)
        else:
            ids, dists = propagate(X, ids, k)
    return ids, dists


# ------------------------------------------------------------------ recall --
def recall(X, ids, k: int, sample, exact=None):
    """Accuracy of Sec. 4 on a sample of points.

    Returns (tie_tolerant, id_set): the first counts a returned neighbour j of
    p when D(p, j) <= D_k(p), the k-th exact distance; the second is
    |returned ids & exact ids| / k.  ``exact`` may pass precomputed
    knn_exact(X, k, sample) output.
    """
    X = _as_f32(X)
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    if exact is None:
        exact = knn_exact(X, k, sample)
    e_ids, e_d = exact
    got = np.asarray(ids)[sample]
    a = np.repeat(sample, k)
    b = got.ravel()
    valid = b >= 0
    dd = np.full(b.shape[0], np.inf)
    if valid.any():
        dd[valid] = pair_dist(X, a[valid], b[valid])
    dd = dd.reshape(-1, k)
    kth = np.array([pair_dist(X, [p], [e_ids[r, -1]])[0] for r, p in enumerate(sample)])
    tie = float(np.mean(np.sum(dd <= kth[:, None], axis=1) / k))
    idset = float(np.mean([len(set(got[r][got[r] >= 0]) & set(e_ids[r])) / k
                           for r in range(len(sample))]))
    return tie, idset
