"""Cosine metric on the GPU, through the C ABI, against the CPU oracle.

The rows are scaled to unit length in FP32 (a fixed summation order, IEEE
sqrt and division), which the oracle states the same way, so the unit rows
and the partitions built on them are bit-exact; the lists follow the FP32
tolerance rule of the L2 path, with distances 1 - cos = |u - v|^2 / 2.
"""
import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic
from test_gpu_parity import assert_valid_rows
from validity import check_build_stagewise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def knng():
    import paper_1307_7852_gb300 as k
    return k


def dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("kind", ["f32_960", "f32_ragged", "f16", "u8"])
def test_normalize_rows_bit_exact(kind):
    rng = np.random.default_rng(7)
    if kind == "f32_960":
        X = synthetic.gist_like(3000, 960, centers=16, seed=2) * np.float32(3.7)
    elif kind == "f32_ragged":
        X = (rng.normal(size=(2000, 37)) * rng.uniform(0.01, 100, size=(2000, 1))).astype(np.float32)
        X[5] = 0.0
    elif kind == "f16":
        X = synthetic.sphere_f16(2000, 96, centers=8, seed=3)
    else:
        X = synthetic.sift_like(2000, 128, centers=8, seed=4).astype(np.uint8)
    U = host(knng().knng_normalize_rows(dev(X)))
    np.testing.assert_array_equal(U, oracle.normalize_rows(X.astype(np.float32)))


def test_partition_of_unit_rows_bit_exact():
    X = synthetic.gaussian_mixture(8000, 64, centers=32, seed=5)
    U = knng().knng_normalize_rows(dev(X))
    perm = host(knng().knng_partition(U, 3, 64, 9))
    Uo = oracle.normalize_rows(X)
    for t in range(3):
        np.testing.assert_array_equal(perm[t], oracle.partition(Uo, 9, t, 64)[0])


@pytest.mark.parametrize("n,d,k,T,g,R", [(6000, 96, 10, 3, 64, 1), (3000, 960, 10, 2, 128, 1), (2500, 30, 8, 4, 40, 2)])
def test_cosine_build_matches_oracle(n, d, k, T, g, R):
    X = synthetic.gaussian_mixture(n, d, centers=24, seed=n + d)
    gi, gd = knng().knng_build(dev(X), k, T, g, R, 11, metric=knng().METRIC_COSINE)
    oi, od = oracle.build_graph(X, k, T, g, R, 11, metric=oracle.METRIC_COSINE)
    gi, gd = host(gi), host(gd)
    assert_valid_rows(gi, gd, n)
    # the build through its stages on the unit rows, every row checked
    check_build_stagewise(knng(), torch, X, k, T, g, R, 11, gi, gd, cosine=True)
    # and against the oracle's whole build where the two agree row for row
    same = np.all(gi == oi, axis=1)
    np.testing.assert_allclose(gd[same], od[same], rtol=1e-5)


def test_cosine_is_scale_invariant_on_gpu():
    X = synthetic.gaussian_mixture(5000, 64, centers=16, seed=8)
    rng = np.random.default_rng(9)
    S = (X * (2.0 ** rng.integers(-8, 9, size=(5000, 1)))).astype(np.float32)
    a = knng().knng_build(dev(X), 10, 3, 64, 1, 2, metric=knng().METRIC_COSINE)
    b = knng().knng_build(dev(S), 10, 3, 64, 1, 2, metric=knng().METRIC_COSINE)
    np.testing.assert_array_equal(host(a[0]), host(b[0]))
    np.testing.assert_array_equal(host(a[1]), host(b[1]))


def test_cosine_on_unit_rows_is_half_the_l2_graph():
    # rows already of unit length up to FP32 rounding: scaling them again
    # changes nothing when they are exactly the FP32 unit rows
    X = oracle.normalize_rows(synthetic.gaussian_mixture(4000, 48, centers=16, seed=10))
    a = knng().knng_build(dev(X), 10, 3, 64, 1, 3, metric=knng().METRIC_COSINE)
    b = knng().knng_build(dev(X), 10, 3, 64, 1, 3)
    Ua = host(knng().knng_normalize_rows(dev(X)))
    if np.array_equal(Ua, X):
        np.testing.assert_array_equal(host(a[0]), host(b[0]))
        np.testing.assert_array_equal(host(a[1]), host(b[1]) * np.float32(0.5))
    else:
        # scaling moved some rows by an FP32 step: the cosine build is still
        # checked in full through its stages
        check_build_stagewise(knng(), torch, X, 10, 3, 64, 1, 3, host(a[0]), host(a[1]), cosine=True)


def test_cosine_batched_and_bf16():
    k = knng()
    Xs = [synthetic.gaussian_mixture(n, 64, centers=8, seed=n) for n in (3000, 5000)]
    outs = k.knng_build_batched([dev(X) for X in Xs], 10, 3, 64, 1, 4, metric=k.METRIC_COSINE)
    for X, (bi, bd) in zip(Xs, outs):
        si, sd = k.knng_build(dev(X), 10, 3, 64, 1, 4, metric=k.METRIC_COSINE)
        np.testing.assert_array_equal(host(bi), host(si))
        np.testing.assert_array_equal(host(bd), host(sd))
    X = Xs[1]
    qi, qd = k.knng_build(dev(X), 10, 3, 64, 1, 4, precision=k.PREC_BF16, metric=k.METRIC_COSINE)
    assert np.all(host(qd) >= 0) and np.all(host(qd) <= 2.0)
    # the BF16 candidate stage on the unit rows, every row checked
    check_build_stagewise(k, torch, X, 10, 3, 64, 1, 4, host(qi), host(qd), precision=k.PREC_BF16, cosine=True)
