"""Tensor-core leaf graphs (tcgen05 Gram in BF16 or FP8 E4M3, FP32 rescoring)
against the CPU oracle, through the C ABI.

The oracle of this stage (a reading of the reduced-precision candidate stage)
takes the k' best by the FP64 distance between the quantised rows, then the k
best of those by the exact distance.  On integer-valued data every bfloat16 is
exact, so the BF16 path must match the exact leaf graph bit for bit.  On
real-valued data the GPU's FP32-accumulated candidate distances can order two
near-equal candidates at the k'-th place differently from FP64; every row is
checked (tests/validity.py): a row may differ from the oracle's only through
candidates whose quantised distance lies within the accumulation error bound
of the k'-th, and its distances must be the pairs' own within 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic

from test_gpu_parity import assert_lists_exact, assert_valid_rows, dev, host, knng
from validity import check_quant_leaf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BF16, FP8 = 1, 2


def _perm(X, T, g, seed):
    Xd = dev(X)
    return Xd, knng().knng_partition(Xd, T, g, seed)


@pytest.mark.parametrize("n,d,k,g", [(10000, 128, 10, 64), (5000, 128, 20, 256), (3000, 100, 8, 512),
                                     (900, 3, 4, 20)])
def test_bf16_integer_data_is_exact(n, d, k, g):
    X = synthetic.sift_like(n, d, centers=16, seed=n + d)
    T = 2
    Xd, perm = _perm(X, T, g, 3)
    ids, dd = knng().knng_leaf_knn(Xd, T, g, perm, k, BF16, 2)
    ids, dd, perm = host(ids), host(dd), host(perm)
    off = knng().knng_leaf_offsets(n, g)
    for t in range(T):
        oi, od = oracle.leaf_knn(X, perm[t], off, k)
        assert_lists_exact(ids[t], dd[t], oi, od)


def _compare_quant(X, T, g, k, mult, prec):
    n = X.shape[0]
    Xd, perm = _perm(X, T, g, 5)
    ids, dd = knng().knng_leaf_knn(Xd, T, g, perm, k, prec, mult)
    ids, dd, perm = host(ids), host(dd), host(perm)
    off = knng().knng_leaf_offsets(n, g)
    assert_valid_rows(ids, dd, n)
    same_rows = 0
    for t in range(T):
        check_quant_leaf(X, perm[t], off, ids[t], dd[t], k, mult * k, prec)
        oi, od = oracle.leaf_knn_quant(X, perm[t], off, k, mult * k, prec)
        same_rows += np.all(ids[t] == oi, axis=1).sum()
    print(f"rows identical to the FP64 quantised oracle: {same_rows / (T * n):.4f}")


@pytest.mark.parametrize("n,d,k,g", [(6000, 96, 10, 128), (3000, 960, 10, 512), (4000, 200, 20, 256)])
def test_bf16_real_valued(n, d, k, g):
    _compare_quant(synthetic.gist_like(n, d, centers=8, seed=n), 2, g, k, 2, BF16)


@pytest.mark.parametrize("n,d,k,g", [(6000, 96, 10, 128), (3000, 960, 10, 512)])
def test_fp8_real_valued(n, d, k, g):
    _compare_quant(synthetic.gist_like(n, d, centers=8, seed=n + 1), 2, g, k, 2, FP8)


def test_fp8_f16_input():
    X = synthetic.sphere_f16(5000, 96, centers=32, seed=30)
    _compare_quant(X, 2, 256, 20, 2, FP8)


def test_bf16_build_integer_matches_oracle():
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    gi, gd = knng().knng_build(dev(X), 10, 4, 64, 1, 7, precision=BF16)
    oi, od = oracle.build_graph(X, 10, 4, 64, 1, 7)
    assert_lists_exact(host(gi), host(gd), oi, od)
    knng().knng_sync()


@pytest.mark.parametrize("k,T,g,R", [(12, 4, 64, 3), (40, 3, 128, 2)])
def test_bf16_build_tree_masks_and_flags_exact(k, T, g, R):
    # exact leaves: the first round skips by the merge's tree masks (k-byte
    # mask rows read per neighbour, four to a word when k is a multiple of
    # 4; two keys per lane when k > 32), later rounds by flags
    X = synthetic.sift_like(8000, 64, centers=32, seed=21)
    gi, gd = knng().knng_build(dev(X), k, T, g, R, 5, precision=BF16)
    oi, od = oracle.build_graph(X, k, T, g, R, 5)
    assert_lists_exact(host(gi), host(gd), oi, od)
    knng().knng_sync()
