"""Byte-valued point rows on the GPU, through the C ABI.

Descriptor data such as SIFT holds integers 0..255.  Such rows may be given
as unsigned bytes (KNNG_DTYPE_U8), and float rows holding only such values
are read from an exact byte copy by the projection and propagation kernels.
Neither may change any result: every stage must equal the one on the equal
float rows, and the whole build must equal the CPU oracle exactly (all
squared distances are integers below 2^24, exact in FP32).
"""
import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic

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


def test_u8_stages_equal_float_stages():
    k = knng()
    Xf = synthetic.sift_like(6000, 128, centers=48, seed=21)
    Xb = Xf.astype(np.uint8)
    T, g, kk, seed = 3, 64, 10, 5
    df, db = dev(Xf), dev(Xb)
    pf, pb = k.knng_partition(df, T, g, seed), k.knng_partition(db, T, g, seed)
    np.testing.assert_array_equal(host(pf), host(pb))
    for prec in (k.PREC_FP32, k.PREC_BF16, k.PREC_FP8E4M3):
        lf = k.knng_leaf_knn(df, T, g, pf, kk, precision=prec)
        lb = k.knng_leaf_knn(db, T, g, pb, kk, precision=prec)
        np.testing.assert_array_equal(host(lf[0]), host(lb[0]))
        np.testing.assert_array_equal(host(lf[1]), host(lb[1]))
    li, ld = k.knng_leaf_knn(df, T, g, pf, kk)
    mi, md = k.knng_merge(li, ld)
    qf = k.knng_propagate(df, mi, md, 2)
    qb = k.knng_propagate(db, mi, md, 2)
    np.testing.assert_array_equal(host(qf[0]), host(qb[0]))
    np.testing.assert_array_equal(host(qf[1]), host(qb[1]))


@pytest.mark.parametrize("dt", ["u8", "f32"])
def test_build_on_bytes_matches_oracle(dt):
    # the 10,000-point SIFT-like workload (k=10, T=4, g=64, R=1), given as
    # bytes or as floats holding bytes (the byte-copy path)
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    Xin = X.astype(np.uint8) if dt == "u8" else X
    gi, gd = knng().knng_build(dev(Xin), 10, 4, 64, 1, 7)
    oi, od = oracle.build_graph(X, 10, 4, 64, 1, 7)
    np.testing.assert_array_equal(host(gi), oi)
    np.testing.assert_array_equal(host(gd), od)


def test_byte_copy_extreme_rows_at_d256():
    # d = 256 with rows of all 0 and all 255: the largest squared distance,
    # 256 * 255^2 = 16,646,400, is still below 2^24
    rng = np.random.default_rng(3)
    X = synthetic.sift_like(3000, 256, centers=16, seed=3)
    X[rng.choice(3000, 20, replace=False)] = 0.0
    X[rng.choice(3000, 20, replace=False)] = 255.0
    gi, gd = knng().knng_build(dev(X), 8, 2, 64, 2, 11)
    oi, od = oracle.build_graph(X, 8, 2, 64, 2, 11)
    np.testing.assert_array_equal(host(gi), oi)
    np.testing.assert_array_equal(host(gd), od)
    assert od[np.isfinite(od)].max() <= 256 * 255 ** 2


@pytest.mark.parametrize("bad", [256.0, -1.0, 17.5, 255.25])
def test_non_byte_entry_disables_the_copy(bad):
    # one entry outside the bytes: the build must read the float rows (an
    # entry read from a byte copy would change that point's distances)
    X = synthetic.sift_like(4000, 64, centers=24, seed=8)
    X[1234, 17] = bad
    gi, gd = knng().knng_build(dev(X), 8, 3, 48, 1, 6)
    oi, od = oracle.build_graph(X, 8, 3, 48, 1, 6)
    gi, gd = host(gi), host(gd)
    np.testing.assert_array_equal(gi, oi)
    np.testing.assert_array_equal(gd, od)


def test_byte_copy_of_strided_rows():
    # float rows with a leading dimension larger than d (a column slice)
    W = synthetic.sift_like(5000, 72, centers=32, seed=12)
    Xd = dev(W)[:, 5:69]
    gi, gd = knng().knng_build(Xd, 10, 3, 64, 2, 13)
    oi, od = oracle.build_graph(np.ascontiguousarray(W[:, 5:69]), 10, 3, 64, 2, 13)
    np.testing.assert_array_equal(host(gi), oi)
    np.testing.assert_array_equal(host(gd), od)


def test_u8_host_entry_point_and_odd_d():
    # d not a multiple of 4: byte rows take the element-wise loads
    X = synthetic.sift_like(2500, 30, centers=12, seed=17)
    hi, hd = knng().knng_build_host(X.astype(np.uint8), 8, 3, 40, 2, 5)
    oi, od = oracle.build_graph(X, 8, 3, 40, 2, 5)
    np.testing.assert_array_equal(hi, oi)
    np.testing.assert_array_equal(hd, od)


@pytest.mark.parametrize("d", [100, 36, 200])
def test_byte_copy_ragged_d(d):
    # d not a multiple of 16: the copy's padding bytes must read as zeros in
    # the 16-byte row loads of projection and propagation
    X = synthetic.sift_like(4000, d, centers=20, seed=d)
    gi, gd = knng().knng_build(dev(X), 10, 3, 64, 2, 3)
    oi, od = oracle.build_graph(X, 10, 3, 64, 2, 3)
    np.testing.assert_array_equal(host(gi), oi)
    np.testing.assert_array_equal(host(gd), od)
