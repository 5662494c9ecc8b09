"""The sift1m configuration at full size (1,000,000 x 128 SIFT-like points,
k = 20, T = 8, leaf size 256, 2 rounds, BF16 leaf Gram), as the benchmark
launches it, against the CPU oracle: one tree's partition in full, the leaf
lists of sampled leaves, the merge in full, and propagation on sampled
points (each stage fed the GPU's previous output); then the whole build
equals the composition of the stages.  Integer data: every comparison is
exact."""
import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, D, K, T, G, R, SEED = 1_000_000, 128, 20, 8, 256, 2, 12345


@pytest.fixture(scope="module")
def data():
    return synthetic.sift_like(N, D, centers=1024, seed=2013)


def test_sift1m_stages_and_build(data):
    import paper_1307_7852_gb300 as k
    X = data
    Xd = torch.from_numpy(X).cuda()
    perm = k.knng_partition(Xd, T, G, SEED)
    li, ld = k.knng_leaf_knn(Xd, T, G, perm, K, precision=k.PREC_BF16)
    mi, md = k.knng_merge(li, ld)
    pi, pd = k.knng_propagate(Xd, mi, md, R)
    gi, gd = k.knng_build(Xd, K, T, G, R, SEED, precision=k.PREC_BF16)
    torch.cuda.synchronize()
    # the build is the composition of the stages, bit for bit
    np.testing.assert_array_equal(gi.cpu().numpy(), pi.cpu().numpy())
    np.testing.assert_array_equal(gd.cpu().numpy(), pd.cpu().numpy())
    perm, li, ld = perm.cpu().numpy(), li.cpu().numpy(), ld.cpu().numpy()
    # tree 0's partition in full
    p0, off = oracle.partition(X, SEED, 0, G)
    np.testing.assert_array_equal(perm[0], p0)
    # leaf lists of 64 sampled leaves of every tree (exact on integer data)
    rng = np.random.default_rng(5)
    for t in range(T):
        leaves = np.sort(rng.choice(len(off) - 1, 64, replace=False))
        sub = np.concatenate([perm[t][off[l]:off[l + 1]] for l in leaves])
        sub_off = np.concatenate([[0], np.cumsum([off[l + 1] - off[l] for l in leaves])])
        oi, od = oracle.leaf_knn(X, sub, sub_off, K)
        np.testing.assert_array_equal(li[t][sub], oi[sub])
        np.testing.assert_array_equal(ld[t][sub], od[sub])
    # the merge in full
    oi, od = oracle.merge(X, li, K)
    mi_h, md_h = mi.cpu().numpy(), md.cpu().numpy()
    np.testing.assert_array_equal(mi_h, oi)
    np.testing.assert_array_equal(md_h, od)
    # two propagation rounds on sampled points, each fed the GPU's input
    q1i, q1d = k.knng_propagate(Xd, mi, md, 1)
    rows = synthetic.sample_ids(N, 3000, 7)
    oi, od = oracle.propagate_rows(X, mi_h, K, rows)
    np.testing.assert_array_equal(q1i.cpu().numpy()[rows], oi)
    np.testing.assert_array_equal(q1d.cpu().numpy()[rows], od)
    q1_h = q1i.cpu().numpy()
    oi, od = oracle.propagate_rows(X, q1_h, K, rows)
    np.testing.assert_array_equal(pi.cpu().numpy()[rows], oi)
    np.testing.assert_array_equal(pd.cpu().numpy()[rows], od)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_maximum_k_trees_and_leaf_size(prec):
    # k = 64, T = 32, leaf size 512 (the library's limits) on integer data
    import paper_1307_7852_gb300 as k
    X = synthetic.sift_like(20000, 64, centers=40, seed=9)
    p = k.PREC_FP32 if prec == "fp32" else k.PREC_BF16
    gi, gd = k.knng_build(torch.from_numpy(X).cuda(), 64, 32, 512, 1, 3, precision=p)
    oi, od = oracle.build_graph(X, 64, 32, 512, 1, 3, precision=p)
    np.testing.assert_array_equal(gi.cpu().numpy(), oi)
    np.testing.assert_array_equal(gd.cpu().numpy(), od)


def test_maximum_d():
    # d = 4096 (the library's limit), real-valued rows: every stage of the
    # build checked in full (tests/validity.py)
    import paper_1307_7852_gb300 as k
    from validity import check_build_stagewise
    X = synthetic.gist_like(1500, 4096, centers=6, seed=3)
    gi, gd = k.knng_build(torch.from_numpy(X).cuda(), 10, 2, 128, 1, 5)
    check_build_stagewise(k, torch, X, 10, 2, 128, 1, 5, gi.cpu().numpy(), gd.cpu().numpy())
