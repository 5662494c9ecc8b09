"""CUDA path vs the CPU oracle, stage by stage (each GPU stage is fed the GPU's
previous-stage output, and the oracle stage is fed the same), through the C ABI.

Bars (arXiv:1307.7852 method; tolerances from the FP32 rescoring):
* partitions: bit-exact canonical leaf sets;
* integer-valued data (SIFT-like): ids and distances exactly equal, ties
  included -- every squared distance is an integer below 2^24, exact in FP32;
* real-valued data: distances within 1e-5 relative of the oracle's FP64 value
  rounded to FP32; ids equal wherever the neighbouring distances differ by
  more than 1e-5 relative.
"""
import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic
from validity import check_build_stagewise, check_quant_leaf, check_rows, merge_candidates, propagation_candidates

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-5


def knng():
    import paper_1307_7852_gb300 as k
    return k


def dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def assert_lists_exact(gi, gd, oi, od):
    np.testing.assert_array_equal(gi, oi)
    np.testing.assert_array_equal(gd, od)


def assert_lists_close(gi, gd, oi, od, rel=REL):
    gi = gi.reshape(-1, gi.shape[-1])
    oi = oi.reshape(-1, oi.shape[-1])
    gd = gd.reshape(gi.shape).astype(np.float64)
    od = od.reshape(oi.shape).astype(np.float64)
    fin = np.isfinite(od)
    assert np.array_equal(np.isfinite(gd), fin)
    tol = rel * np.maximum(np.abs(od[fin]), 1e-30)
    assert np.all(np.abs(gd[fin] - od[fin]) <= tol), np.max(np.abs(gd[fin] - od[fin]) / np.maximum(od[fin], 1e-30))
    k = od.shape[1]
    left = np.full(od.shape, np.inf)
    left[:, 1:] = (od[:, 1:] - od[:, :-1]) / np.maximum(od[:, 1:], 1e-30)
    right = np.full(od.shape, np.inf)
    right[:, :-1] = (od[:, 1:] - od[:, :-1]) / np.maximum(od[:, 1:], 1e-30)
    right[:, k - 1] = 0.0  # the next oracle candidate is not visible: the last slot may tie
    iso = (left > rel) & (right > rel)
    mism = iso & (gi != oi)
    assert not mism.any(), f"{mism.sum()} isolated positions differ"


def assert_valid_rows(ids, dists, n):
    k = ids.shape[-1]
    ids = ids.reshape(-1, k)
    dists = dists.reshape(-1, k)
    assert np.all((ids >= -1) & (ids < n))
    d64 = dists.astype(np.float64)
    assert np.all(np.diff(np.where(np.isfinite(d64), d64, np.inf), axis=1) >= 0)
    for r in range(0, ids.shape[0], max(1, ids.shape[0] // 500)):
        v = ids[r][ids[r] >= 0]
        assert len(np.unique(v)) == len(v)


# ------------------------------------------------------------- partitions --
PART_CASES = [
    # (name, X-maker, T, g, seed)
    ("sift10k", lambda: synthetic.sift_like(10000, 128, centers=64, seed=1), 4, 64, 7),
    ("ragged_d3", lambda: synthetic.gist_like(3001, 3, centers=5, seed=2), 3, 50, 11),
    ("dups", lambda: np.random.default_rng(3).integers(0, 2, size=(2000, 4)).astype(np.float32), 2, 16, 5),
    ("multiblock", lambda: synthetic.sift_like(40000, 20, centers=32, seed=4), 2, 40, 3),
    ("single_leaf", lambda: synthetic.sift_like(300, 16, centers=4, seed=5), 2, 512, 1),
    ("d960", lambda: synthetic.gist_like(6000, 960, centers=16, seed=6), 2, 512, 2),
]


@pytest.mark.parametrize("name,mk,T,g,seed", PART_CASES, ids=[c[0] for c in PART_CASES])
def test_partition_bit_exact(name, mk, T, g, seed):
    X = mk()
    perm = host(knng().knng_partition(dev(X), T, g, seed))
    off = knng().knng_leaf_offsets(X.shape[0], g)
    for t in range(T):
        op, oo = oracle.partition(X, seed, t, g)
        np.testing.assert_array_equal(off, oo)
        np.testing.assert_array_equal(perm[t], op)


def test_partition_f16_and_strided():
    X16 = synthetic.sphere_f16(5000, 96, centers=32, seed=8)
    perm = host(knng().knng_partition(dev(X16), 2, 64, 9))
    for t in range(2):
        np.testing.assert_array_equal(perm[t], oracle.partition(X16, 9, t, 64)[0])
    # rows with a leading dimension larger than d (a column slice)
    W = synthetic.sift_like(3000, 40, centers=8, seed=10)
    Xd = dev(W)[:, 3:35]
    perm = host(knng().knng_partition(Xd, 2, 32, 4))
    for t in range(2):
        np.testing.assert_array_equal(perm[t], oracle.partition(W[:, 3:35], 4, t, 32)[0])


# ------------------------------------------------------------- leaf graph --
def test_leaf_knn_integer_exact():
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    k, T, g = 10, 4, 64
    Xd = dev(X)
    perm = knng().knng_partition(Xd, T, g, 7)
    ids, dd = knng().knng_leaf_knn(Xd, T, g, perm, k)
    ids, dd, perm = host(ids), host(dd), host(perm)
    off = knng().knng_leaf_offsets(10000, g)
    for t in range(T):
        oi, od = oracle.leaf_knn(X, perm[t], off, k)
        assert_lists_exact(ids[t], dd[t], oi, od)


@pytest.mark.parametrize("n,d,k,g", [(4000, 50, 7, 40), (3000, 200, 20, 256), (1500, 960, 10, 512), (700, 33, 5, 12)])
def test_leaf_knn_real_valued(n, d, k, g):
    # the FP32 Gram selects 2k candidates, rescored exactly: every row is the
    # exact top-k of its leaf unless a candidate within the FP32 Gram's error
    # bound of the 2k-th was exchanged (tests/validity.py)
    X = synthetic.gist_like(n, d, centers=8, seed=n + d)
    T = 2
    Xd = dev(X)
    perm = knng().knng_partition(Xd, T, g, 3)
    ids, dd = knng().knng_leaf_knn(Xd, T, g, perm, k)
    ids, dd, perm = host(ids), host(dd), host(perm)
    off = knng().knng_leaf_offsets(n, g)
    for t in range(T):
        check_quant_leaf(X, perm[t], off, ids[t], dd[t], k, 2 * k, oracle.PREC_FP32)
    assert_valid_rows(ids, dd, n)


def test_leaf_knn_padding_small_n():
    X = synthetic.sift_like(6, 8, centers=2, seed=12)
    Xd = dev(X)
    perm = knng().knng_partition(Xd, 1, 64, 1)
    ids, dd = knng().knng_leaf_knn(Xd, 1, 64, perm, 9)
    ids, dd = host(ids)[0], host(dd)[0]
    oi, od = oracle.leaf_knn(X, host(perm)[0], knng().knng_leaf_offsets(6, 64), 9)
    assert_lists_exact(ids, dd, oi, od)
    assert np.all(ids[:, 5:] == -1)


# ------------------------------------------------------------------ merge --
def _gpu_leaf_lists(X, T, g, k, seed):
    Xd = dev(X)
    perm = knng().knng_partition(Xd, T, g, seed)
    return Xd, knng().knng_leaf_knn(Xd, T, g, perm, k)


def test_merge_integer_exact():
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    Xd, (li, ld) = _gpu_leaf_lists(X, 4, 64, 10, 7)
    mi, md = knng().knng_merge(li, ld)
    oi, od = oracle.merge(X, host(li), 10)
    assert_lists_exact(host(mi), host(md), oi, od)


def test_merge_real_valued():
    X = synthetic.gist_like(5000, 64, centers=16, seed=13)
    Xd, (li, ld) = _gpu_leaf_lists(X, 5, 48, 8, 2)
    mi, md = knng().knng_merge(li, ld)
    oi, od = oracle.merge(X, host(li), 8)
    check_rows(X, host(mi), host(md), oi, od, cands=merge_candidates(host(li)))


# ------------------------------------------------------------ propagation --
def test_propagate_integer_exact():
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    Xd, (li, ld) = _gpu_leaf_lists(X, 4, 64, 10, 7)
    mi, md = knng().knng_merge(li, ld)
    pi, pd = knng().knng_propagate(Xd, mi, md, 1)
    oi, od = oracle.propagate(X, host(mi), 10)
    assert_lists_exact(host(pi), host(pd), oi, od)
    # a second round, again fed the GPU's own previous output
    qi, qd = knng().knng_propagate(Xd, pi, pd, 1)
    oi2, od2 = oracle.propagate(X, host(pi), 10)
    assert_lists_exact(host(qi), host(qd), oi2, od2)
    # never worsens any list
    assert np.all(host(qd) <= host(pd)) and np.all(host(pd) <= host(md))


def test_propagate_rounds_skip_old_pairs():
    # three rounds in one call: rounds 2 and 3 skip the pairs the previous
    # round already scored; the result must equal three plain oracle rounds
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    Xd, (li, ld) = _gpu_leaf_lists(X, 2, 64, 10, 9)
    mi, md = knng().knng_merge(li, ld)
    pi, pd = knng().knng_propagate(Xd, mi, md, 3)
    oi = host(mi)
    for _ in range(3):
        oi, od = oracle.propagate(X, oi, 10)
    assert_lists_exact(host(pi), host(pd), oi, od)


@pytest.mark.parametrize("n,d,k", [(6000, 96, 16), (2500, 7, 40)])
def test_propagate_real_valued(n, d, k):
    X = synthetic.gist_like(n, d, centers=16, seed=n)
    g = max(2 * k + 2, 96)
    Xd, (li, ld) = _gpu_leaf_lists(X, 3, g, k, 4)
    mi, md = knng().knng_merge(li, ld)
    pi, pd = knng().knng_propagate(Xd, mi, md, 1)
    oi, od = oracle.propagate(X, host(mi), k)
    check_rows(X, host(pi), host(pd), oi, od, cands=propagation_candidates(host(mi)))
    assert_valid_rows(host(pi), host(pd), n)


# ------------------------------------------------------------ whole method --
def test_build_matches_oracle_on_integer_data():
    # the 10,000-point SIFT-like workload: k=10, T=4, g=64, R=1
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    gi, gd = knng().knng_build(dev(X), 10, 4, 64, 1, 7)
    oi, od = oracle.build_graph(X, 10, 4, 64, 1, 7)
    assert_lists_exact(host(gi), host(gd), oi, od)


def test_build_host_entry_point():
    X = synthetic.sift_like(3000, 32, centers=16, seed=14)
    hi, hd = knng().knng_build_host(X, 8, 3, 40, 2, 5)
    gi, gd = knng().knng_build(dev(X), 8, 3, 40, 2, 5)
    np.testing.assert_array_equal(hi, host(gi))
    np.testing.assert_array_equal(hd, host(gd))


def test_build_f16_input():
    # real-valued FP16 rows: the build is checked through its stages, each
    # fed the GPU's previous output, every row complete (tests/validity.py)
    X = synthetic.sphere_f16(4000, 96, centers=32, seed=15)
    gi, gd = knng().knng_build(dev(X), 10, 3, 64, 1, 2)
    gi, gd = host(gi), host(gd)
    assert_valid_rows(gi, gd, 4000)
    check_build_stagewise(knng(), torch, X, 10, 3, 64, 1, 2, gi, gd)


def test_invalid_arguments_are_rejected():
    k = knng()
    X = dev(synthetic.sift_like(100, 8, centers=2, seed=1))
    with pytest.raises(k.KnngError) as e:
        k.knng_build(X, 40, 2, 64, 0, 1)  # k >= leaf_size / 2
    assert e.value.code == -1
    with pytest.raises(k.KnngError):
        k.knng_build(X, 4, 0, 64, 0, 1)  # T = 0
    with pytest.raises(k.KnngError):
        k.knng_build(X, 4, 2, 1024, 0, 1)  # leaf size above 512


# ------------------------------------------------------- exact k-NN (recall)
def test_exact_knn_matches_oracle():
    X = synthetic.sift_like(5000, 64, centers=8, seed=20)
    q = synthetic.sample_ids(5000, 300, 3)
    gi, gd = knng().knng_exact_knn(dev(X), dev(q), 12)
    oi, od = oracle.knn_exact(X, 12, q)
    assert_lists_exact(host(gi), host(gd), oi, od)
    Y = synthetic.gist_like(4000, 130, centers=8, seed=21)
    q = synthetic.sample_ids(4000, 200, 4)
    gi, gd = knng().knng_exact_knn(dev(Y), dev(q), 33)
    oi, od = oracle.knn_exact(Y, 33, q)
    check_rows(Y, host(gi), host(gd), oi, od, rows=q)
