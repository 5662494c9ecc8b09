"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks one oracle function against a published value, a closed
form, an exact special case, an independent NumPy brute force on tiny inputs,
or an invariant of the method (Sec. 3 of arXiv:1307.7852).  No GPU needed.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ helpers (numpy)
def np_sqdist(X, i, J):
    X = X.astype(np.float64)
    diff = X[J] - X[i][None, :]
    return np.einsum("ij,ij->i", diff, diff)


def np_topk(D, ids, k):
    """k smallest by (D, id); pads with (-1, inf)."""
    order = np.lexsort((ids, D))[:k]
    out_i = np.full(k, -1, dtype=np.int64)
    out_d = np.full(k, np.inf)
    out_i[:len(order)] = ids[order]
    out_d[:len(order)] = D[order]
    return out_i, out_d


def np_knn_exact(X, k):
    n = X.shape[0]
    ids = np.empty((n, k), dtype=np.int64)
    dd = np.empty((n, k))
    allj = np.arange(n)
    for i in range(n):
        J = allj[allj != i]
        ids[i], dd[i] = np_topk(np_sqdist(X, i, J), J, k)
    return ids, dd


def tiny_ints(n, d, seed, hi=8):
    rng = np.random.default_rng(seed)
    return rng.integers(0, hi, size=(n, d)).astype(np.float32)


# ------------------------------------------------------------------ Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(h, 16) for h in r]
        got = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in got] == v[6:10]


# --------------------------------------------------------------- directions
def _tri(u):
    return ((u & 0xFFFF) + (u >> 16) - 65535) / 65536.0


def test_direction_zero_counter_is_kat_words():
    # seed 0, tree 0, level 0, node 0 uses counter (0,0,0,0) and key (0,0):
    # the first published known-answer vector.
    words = [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    a = oracle.direction(0, 0, 0, 0, 4)
    assert [float(x) for x in a] == [_tri(w) for w in words]
    # hand value of the first entry: 0xe8d5 + 0x6627 - 65535 = 20221
    assert float(a[0]) == 20221 / 65536.0


def test_direction_values_and_law():
    vals = np.concatenate([oracle.direction(7, t, lvl, v, 256)
                           for t in range(4) for lvl in range(3) for v in range(8)])
    scaled = vals.astype(np.float64) * 65536.0
    assert np.all(scaled == np.rint(scaled))          # multiples of 2^-16
    assert np.all(np.abs(vals) < 1.0)
    # triangular law of (U1 + U2 - 65535) / 65536, U uniform on 0..65535:
    # mean 0, variance 2 * (65536^2 - 1) / 12 / 65536^2 ~= 1/6
    assert abs(vals.mean()) < 0.01
    assert abs(vals.var() - 1.0 / 6.0) < 0.01
    # distinct nodes, levels, trees and seeds give distinct directions
    a = oracle.direction(7, 0, 1, 0, 64)
    assert not np.array_equal(a, oracle.direction(7, 0, 1, 1, 64))
    assert not np.array_equal(a, oracle.direction(7, 1, 1, 0, 64))
    assert not np.array_equal(a, oracle.direction(8, 0, 1, 0, 64))
    assert not np.array_equal(a, oracle.direction(7, 0, 2, 0, 64))


# --------------------------------------------------------------- projection
def test_projection_exact_small_cases():
    # small integers times multiples of 2^-16 with few terms: every product and
    # partial sum is exact in FP32, so the projection equals the exact dot.
    rng = np.random.default_rng(1)
    for d in (1, 2, 3, 4, 5, 7, 16):
        for _ in range(20):
            x = rng.integers(0, 4, size=d).astype(np.float32)
            a = oracle.direction(int(rng.integers(1 << 30)), 0, 0, 0, d)
            exact = float(np.dot(x.astype(np.float64), a.astype(np.float64)))
            assert float(oracle.project(x, a)) == exact


def test_projection_lane_order():
    # lane 0 owns x0..x3 and lane 1 owns x4..x7: lane sums 2^25 and 4 add
    # exactly; a sequential or lane-strided order loses the three 1s.
    x = np.array([2.0 ** 25, 0, 0, 0, 1, 1, 1, 1], dtype=np.float32)
    a = np.ones(8, dtype=np.float32)
    assert float(oracle.project(x, a)) == 2.0 ** 25 + 4


def test_projection_error_bound():
    rng = np.random.default_rng(2)
    for d in (17, 128, 300, 960):
        for _ in range(10):
            x = rng.normal(size=d).astype(np.float32)
            a = oracle.direction(int(rng.integers(1 << 30)), 1, 2, 3, d)
            s = float(oracle.project(x, a))
            xa = x.astype(np.float64) * a.astype(np.float64)
            terms = 4 * ((d + 127) // 128) + 5
            bound = 1.01 * terms * 2.0 ** -24 * np.abs(xa).sum()
            assert abs(s - xa.sum()) <= bound


def test_ord_is_monotone():
    v = np.array([-np.inf, -3e38, -1.5, -1e-40, 0.0, 1e-40, 1.0, 2.5, 3e38, np.inf],
                 dtype=np.float32)
    o = [oracle.ord32(float(x)) for x in v]
    assert all(o[i] < o[i + 1] for i in range(len(o) - 1))
    assert oracle.ord32(0.0) == 0x80000000
    assert oracle.ord32(-1.5) == (~np.float32(-1.5).view(np.uint32)).item()


# ---------------------------------------------------------------- partition
def _expected_leaves_1d(x, seed, t, g):
    """Independent restatement for d = 1: a node sorts its members by x times
    the sign of its direction (ties by id), gives the first floor(m/2) to
    child 2v and the rest to 2v+1, and stops at m <= g."""
    leaves = []

    def rec(ids, level, v):
        if len(ids) <= g:
            leaves.append(sorted(ids))
            return
        a0 = float(oracle.direction(seed, t, level, v, 1)[0])
        key = [(x[i] * a0, i) for i in ids]
        order = [i for _, i in sorted(key)]
        m = len(ids)
        rec(order[:m // 2], level + 1, 2 * v)
        rec(order[m // 2:], level + 1, 2 * v + 1)

    rec(list(range(len(x))), 0, 0)
    return leaves


@pytest.mark.parametrize("n,g", [(64, 8), (100, 7), (127, 16), (33, 2)])
def test_partition_1d_is_sorting(n, g):
    rng = np.random.default_rng(n + g)
    x = rng.permutation(n).astype(np.float32)  # distinct, x * a exact in FP32
    for t in range(3):
        perm, off = oracle.partition(x[:, None], 11, t, g)
        got = [list(perm[off[i]:off[i + 1]]) for i in range(len(off) - 1)]
        assert got == _expected_leaves_1d(x, 11, t, g)


def test_partition_structure():
    X = synthetic.sift_like(3000, 32, centers=16, seed=3)
    for g in (8, 64, 5000):
        perm, off = oracle.partition(X, 5, 0, g)
        assert sorted(perm.tolist()) == list(range(3000))
        sizes = np.diff(off)
        assert len(sizes) == oracle.leaf_count(3000, g)
        if g < 3000:
            assert sizes.min() >= (g + 1) // 2 and sizes.max() <= g
        else:
            assert sizes.tolist() == [3000]
        for i in range(len(sizes)):
            seg = perm[off[i]:off[i + 1]]
            assert np.all(np.diff(seg) > 0)  # canonical: ids ascending


def test_leaf_count_closed_form():
    # floor/ceil halving keeps the sizes at level l in {floor(n/2^l),
    # ceil(n/2^l)}; with h the first level whose ceil size is <= g, every
    # leaf sits at depth h when floor(n/2^(h-1)) > g, else at h-1 or h.
    for n, g in [(10000, 64), (1000000, 256), (1000000, 512), (10000000, 256),
                 (5, 8), (300, 150), (301, 150), (1000, 3)]:
        h = 0
        while -(-n // (1 << h)) > g:
            h += 1
        cnt = oracle.leaf_count(n, g)
        if h == 0 or n // (1 << (h - 1)) > g:
            assert cnt == 1 << h
        else:
            assert (1 << (h - 1)) < cnt < (1 << h)


# --------------------------------------------------------------- leaf graph
def test_leaf_knn_is_brute_force_per_leaf():
    X = tiny_ints(300, 6, 4)  # many exact ties: exercises the id tie-break
    k = 5
    perm, off = oracle.partition(X, 9, 1, 40)
    ids, dd = oracle.leaf_knn(X, perm, off, k)
    for L in range(len(off) - 1):
        mem = perm[off[L]:off[L + 1]]
        for i in mem:
            J = mem[mem != i]
            ei, ed = np_topk(np_sqdist(X, i, J), J, k)
            assert ids[i].tolist() == ei.tolist()
            assert np.array_equal(dd[i], ed.astype(np.float32))


def test_single_leaf_is_exact_knn_and_padding():
    X = tiny_ints(60, 5, 5)
    perm, off = oracle.partition(X, 1, 0, 64)
    ids, dd = oracle.leaf_knn(X, perm, off, 7)
    ei, ed = np_knn_exact(X, 7)
    assert np.array_equal(ids, ei)
    assert np.array_equal(dd, ed.astype(np.float32))
    # fewer than k other points: padded with (-1, +inf)
    Xs = X[:5]
    perm, off = oracle.partition(Xs, 1, 0, 8)
    ids, dd = oracle.leaf_knn(Xs, perm, off, 6)
    assert np.all(ids[:, 4:] == -1) and np.all(np.isinf(dd[:, 4:]))
    assert np.all(ids[:, :4] >= 0)


def test_knn_exact_matches_numpy():
    X = tiny_ints(200, 4, 6, hi=4)  # heavy ties
    ids, dd = oracle.knn_exact(X, 9)
    ei, ed = np_knn_exact(X, 9)
    assert np.array_equal(ids, ei)
    assert np.array_equal(dd, ed.astype(np.float32))
    q = np.array([3, 50, 199], dtype=np.int32)
    qi, qd = oracle.knn_exact(X, 9, q)
    assert np.array_equal(qi, ei[q])


# -------------------------------------------------------------------- merge
def _lists(X, T, g, k, seed):
    out = []
    for t in range(T):
        perm, off = oracle.partition(X, seed, t, g)
        out.append(oracle.leaf_knn(X, perm, off, k)[0])
    return np.stack(out)


def test_merge_is_topk_of_union():
    X = tiny_ints(400, 8, 7)
    k = 6
    L = _lists(X, 3, 30, k, 2)
    ids, dd = oracle.merge(X, L, k)
    for p in range(0, 400, 7):
        U = np.unique(L[:, p, :])
        U = U[(U >= 0) & (U != p)]
        ei, ed = np_topk(np_sqdist(X, p, U), U, k)
        assert ids[p].tolist() == ei.tolist()
        assert np.array_equal(dd[p], ed.astype(np.float32))
    # one tree: the merge returns the tree's own list
    one, _ = oracle.merge(X, L[:1], k)
    assert np.array_equal(one, L[0])


def test_merge_recall_never_decreases_with_T():
    # tree t depends only on (seed, t): the candidate set for T+1 trees
    # contains the one for T, so the per-point tie-tolerant recall of the
    # (D, id) top-k cannot drop.
    X = synthetic.sift_like(2000, 16, centers=8, std=20.0, seed=8)
    k = 8
    exact_i, exact_d = oracle.knn_exact(X, k)
    kth = exact_d[:, -1].astype(np.float64)
    L = _lists(X, 5, 32, k, 4)
    prev = None
    for T in range(1, 6):
        ids, dd = oracle.merge(X, L[:T], k)
        # per-point number of returned neighbours inside the exact k-ball
        hits = np.sum(dd.astype(np.float64) <= kth[:, None], axis=1)
        if prev is not None:
            assert np.all(hits >= prev)
        prev = hits
    assert prev.mean() > 0


# ---------------------------------------------------------------- propagate
def test_propagation_never_worsens_and_is_candidate_subset():
    X = synthetic.sift_like(1500, 16, centers=8, seed=9)
    k = 6
    L = _lists(X, 2, 32, k, 5)
    ids, dd = oracle.merge(X, L, k)
    for _ in range(2):
        nid, ndd = oracle.propagate(X, ids, k)
        assert np.all(ndd <= dd)
        for p in range(0, 1500, 37):
            cand = set(ids[p]) | set(ids[ids[p]].ravel())
            cand.discard(p)
            cand.discard(-1)
            assert set(nid[p]) <= cand
            assert len(set(nid[p])) == k and p not in nid[p]
        ids, dd = nid, ndd


def test_propagation_fixed_point_on_exact_graph():
    X = tiny_ints(250, 5, 10)
    ei, ed = oracle.knn_exact(X, 6)
    pi, pd = oracle.propagate(X, ei, 6)
    assert np.array_equal(pi, ei) and np.array_equal(pd, ed)


def test_propagation_matches_numpy():
    X = tiny_ints(200, 6, 11)
    k = 4
    L = _lists(X, 1, 16, k, 6)
    ids, _ = oracle.merge(X, L, k)
    pi, pd = oracle.propagate(X, ids, k)
    for p in range(200):
        C = np.unique(np.concatenate([ids[p], ids[ids[p]].ravel()]))
        C = C[(C >= 0) & (C != p)]
        ei, ed = np_topk(np_sqdist(X, p, C), C, k)
        assert pi[p].tolist() == ei.tolist()


# ------------------------------------------------------------- precision
def test_bf16_rounding_matches_library():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    v = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-30, 30, size=2000),
                        np.float32(1.0) + np.arange(0, 64) * np.float32(2.0 ** -9)]).astype(np.float32)
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    got = np.array([oracle.bf16_round(float(x)) for x in v], dtype=np.float32)
    assert np.array_equal(got, want)
    assert oracle.bf16_round(1.0 + 2.0 ** -8) == 1.0          # tie -> even
    assert oracle.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


def test_e4m3_rounding_matches_library():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(13)
    v = np.concatenate([rng.uniform(-463.0, 463.0, 3000),
                        rng.normal(size=2000) * 2.0 ** rng.integers(-12, 4, size=2000)]).astype(np.float32)
    want = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    got = np.array([oracle.e4m3_round(float(x)) for x in v], dtype=np.float32)
    assert np.array_equal(got, want)
    assert oracle.e4m3_round(1.0625) == 1.0      # tie -> even mantissa
    assert oracle.e4m3_round(1.1875) == 1.25
    assert oracle.e4m3_round(470.0) == 448.0     # saturates to the largest finite
    assert oracle.e4m3_round(-1e9) == -448.0
    assert oracle.e4m3_round(2.0 ** -10) == 0.0  # half the smallest subnormal


def test_quantized_rows():
    X = synthetic.gist_like(50, 64, centers=4, seed=14)
    q, s = oracle.quantize_rows(X, oracle.PREC_FP8E4M3)
    mx = np.abs(X).max(axis=1)
    assert np.array_equal(s, (mx / np.float32(448.0)).astype(np.float32))
    # the largest entry of each row lands on (or saturates to) code 448
    r = np.arange(50)
    j = np.abs(X).argmax(axis=1)
    assert np.allclose(q[r, j] / s.astype(np.float64), 448.0)
    # relative error of E4M3 codes is at most 2^-4 in the normal range
    big = np.abs(X) / s[:, None] >= 2.0 ** -6
    rel = np.abs(q - X.astype(np.float64))[big] / np.abs(X.astype(np.float64))[big]
    assert rel.max() <= 2.0 ** -4 + 1e-12
    qb, _ = oracle.quantize_rows(X, oracle.PREC_BF16)
    relb = np.abs(qb - X)[X != 0] / np.abs(X)[X != 0]
    assert relb.max() <= 2.0 ** -8 + 1e-12


def test_bf16_candidate_stage_exact_on_integer_data():
    # integers 0..255 are exact in bfloat16, so the reduced-precision
    # candidate stage sees the exact distances and changes nothing
    X = synthetic.sift_like(800, 24, centers=8, seed=15)
    perm, off = oracle.partition(X, 3, 0, 64)
    a = oracle.leaf_knn(X, perm, off, 5)
    b = oracle.leaf_knn_quant(X, perm, off, 5, 10, oracle.PREC_BF16)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_candidate_stage_keeping_all_is_exact():
    X = synthetic.gist_like(500, 32, centers=4, seed=16)
    perm, off = oracle.partition(X, 3, 0, 40)
    a = oracle.leaf_knn(X, perm, off, 4)
    b = oracle.leaf_knn_quant(X, perm, off, 4, 64, oracle.PREC_FP8E4M3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# -------------------------------------------------------------- whole method
def test_build_single_leaf_is_exact():
    X = tiny_ints(120, 6, 17)
    ids, dd = oracle.build_graph(X, 5, 3, 200, 1, 4)
    ei, ed = oracle.knn_exact(X, 5)
    assert np.array_equal(ids, ei)


def test_build_recall_grows_with_trees_and_propagation():
    X = synthetic.sift_like(4000, 32, centers=16, seed=18)
    k = 10
    sample = synthetic.sample_ids(4000, 300, 1)
    exact = oracle.knn_exact(X, k, sample)
    r1 = oracle.recall(X, oracle.build_graph(X, k, 1, 64, 0, 2)[0], k, sample, exact)[0]
    r4 = oracle.recall(X, oracle.build_graph(X, k, 4, 64, 0, 2)[0], k, sample, exact)[0]
    r4p = oracle.recall(X, oracle.build_graph(X, k, 4, 64, 1, 2)[0], k, sample, exact)[0]
    assert r1 < r4 < r4p <= 1.0


# ------------------------------------------------------------ cosine metric --
def test_normalize_rows_pins():
    rng = np.random.default_rng(41)
    X = rng.normal(size=(300, 37)).astype(np.float32)
    X[7] = 0.0
    U = oracle.normalize_rows(X)
    nrm = np.linalg.norm(U.astype(np.float64), axis=1)
    live = np.ones(300, bool)
    live[7] = False
    assert np.all(np.abs(nrm[live] - 1.0) < 4e-7)
    assert np.all(U[7] == 0.0)
    # each entry is the FP32 rounding of x_j / |x| up to the rounding of |x|
    ref = X.astype(np.float64) / np.linalg.norm(X.astype(np.float64), axis=1, keepdims=True).clip(1e-300)
    assert np.max(np.abs(U[live] - ref[live]) / np.abs(ref[live]).clip(1e-30)) < 3e-7
    # scaling a row by a power of two leaves its unit row bit-identical
    S = X * (2.0 ** rng.integers(-20, 20, size=(300, 1))).astype(np.float32)
    np.testing.assert_array_equal(oracle.normalize_rows(S), U)


def test_cosine_graph_is_brute_force_cosine_on_one_leaf():
    # one leaf holding every point (g >= n), no propagation: the cosine
    # graph must be the textbook one, 1 - x.y / (|x| |y|) in FP64
    rng = np.random.default_rng(42)
    n, d, k = 250, 24, 9
    X = (rng.normal(size=(n, d)) * rng.uniform(0.1, 10.0, size=(n, 1))).astype(np.float32)
    ids, dists = oracle.build_graph(X, k, 1, 256, 0, 3, metric=oracle.METRIC_COSINE)
    Xd = X.astype(np.float64)
    nx = np.linalg.norm(Xd, axis=1)
    C = 1.0 - (Xd @ Xd.T) / np.outer(nx, nx)
    np.fill_diagonal(C, np.inf)
    want = np.argsort(C, axis=1, kind="stable")[:, :k]
    np.testing.assert_array_equal(ids, want)
    np.testing.assert_allclose(dists, np.take_along_axis(C, want, axis=1), rtol=2e-6)


def test_cosine_graph_is_scale_invariant():
    X = synthetic.gist_like(1500, 40, centers=12, seed=5)
    rng = np.random.default_rng(43)
    S = (X * (2.0 ** rng.integers(-6, 7, size=(1500, 1)))).astype(np.float32)
    a = oracle.build_graph(X, 8, 2, 48, 1, 4, metric=oracle.METRIC_COSINE)
    b = oracle.build_graph(S, 8, 2, 48, 1, 4, metric=oracle.METRIC_COSINE)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_propagate_rows_is_the_round_on_those_rows():
    X = synthetic.sift_like(3000, 32, centers=8, seed=1)
    ids, _ = oracle.build_graph(X, 8, 2, 40, 0, 3)
    full = oracle.propagate(X, ids, 8)
    rows = np.array([5, 17, 2999, 0, 1500])
    part = oracle.propagate_rows(X, ids, 8, rows)
    np.testing.assert_array_equal(part[0], full[0][rows])
    np.testing.assert_array_equal(part[1], full[1][rows])
