"""Learned partitioner on the GPU, through the C ABI: training gradients
against the FP64 oracle, BF16 inference against the FP64 forward pass, the
training loop, persistence, and what the trained network gains over random
directions at an equal number of trees."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1307_7852_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAM, EPS = 0.05, 1e-4


def knng():
    import paper_1307_7852_gb300 as k
    return k


def test_gradients_match_fp64_oracle():
    k = knng()
    net = k.Mlp(96, 256, 16, seed=3)
    rng = np.random.default_rng(0)
    B = 512
    Xi = rng.normal(size=(B, 96)).astype(np.float32)
    Xj = (Xi + 0.3 * rng.normal(size=(B, 96))).astype(np.float32)
    Xp = np.concatenate([Xi, Xj])
    loss, g = net.loss_grad(torch.from_numpy(Xp).cuda())
    W1, b1, W2, b2 = net.get_params()
    L, (gW1, gb1, gW2, gb2) = omlp.loss_and_grads(Xp, W1, b1, W2, b2, lam=LAM, eps=EPS)
    g = g.cpu().numpy().astype(np.float64)
    want = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2])
    assert abs(loss - L) <= 1e-4 * abs(L)
    scale = np.abs(want).max()
    assert np.max(np.abs(g - want)) <= 2e-3 * scale, np.max(np.abs(g - want)) / scale
    # per block: relative error small, measured against the block or, for a
    # block that vanishes analytically, against the whole gradient
    o = 0
    total = np.linalg.norm(want)
    for part in (gW1, gb1, gW2, gb2):
        sz = part.size
        err = np.linalg.norm(g[o:o + sz] - part.ravel())
        assert err <= 1e-3 * np.linalg.norm(part) + 1e-5 * total, (err, np.linalg.norm(part), total)
        o += sz


def test_bf16_inference_matches_fp64_forward():
    k = knng()
    net = k.Mlp(96, 256, 16, seed=5)
    X = synthetic.sphere_f16(3000, 96, centers=16, seed=2)
    Z = k.knng_mlp_forward(net, torch.from_numpy(X).cuda()).cpu().numpy()
    _, _, Zr = omlp.forward(X.astype(np.float64), *net.get_params())
    # BF16 inputs, weights and hidden activations: errors of a few 2^-8
    # relative to the spread of each output
    err = np.abs(Z - Zr) / Zr.std(axis=0)
    assert np.percentile(err, 99) < 0.05 and err.max() < 0.2
    assert np.corrcoef(Z.ravel(), Zr.ravel())[0, 1] > 0.999


def test_training_lowers_the_loss_and_persists(tmp_path):
    k = knng()
    X = torch.from_numpy(synthetic.sphere_f16(20000, 96, centers=64, seed=3)).cuda()
    ids, _ = k.knng_build(X, 10, 4, 128, 1, 1)
    net = k.Mlp(96, 256, 16, seed=1)
    first = net.train(X, ids, 1, batch_edges=2048, lr=1e-3, seed=5)
    last = net.train(X, ids, 300, batch_edges=2048, lr=1e-3, seed=6)
    assert last < 0.7 * first, (first, last)
    path = str(tmp_path / "net.bin")
    net.save(path)
    other = k.Mlp(96, 256, 16, seed=99)
    other.load(path)
    for a, b in zip(net.get_params(), other.get_params()):
        np.testing.assert_array_equal(a, b)


def _recall(X, ids, k, sample):
    Xd = torch.from_numpy(X).cuda()
    q = torch.from_numpy(sample).cuda()
    import paper_1307_7852_gb300 as kk
    ei, ed = kk.knng_exact_knn(Xd, q, k)
    gi = ids[q.long()].cpu().numpy()
    e = ei.cpu().numpy()
    return float(np.mean([len(set(gi[r]) & set(e[r])) / k for r in range(len(sample))]))


@pytest.fixture(scope="module")
def trained():
    k = knng()
    n, d, kk = 60000, 96, 20
    X = synthetic.sphere_f16(n, d, centers=256, std=0.05, seed=11)
    # training graph: the method itself, random directions, on a subsample
    sub = torch.from_numpy(np.ascontiguousarray(X[: n // 2])).cuda()
    gi, _ = k.knng_build(sub, kk, 8, 256, 1, 7)
    net = k.Mlp(d, 256, 16, seed=2)
    net.train(sub, gi, 600, batch_edges=4096, lr=2e-3, seed=3)
    return X, net


@pytest.mark.parametrize("mode", ["embedding_random", "features"])
def test_learned_splits_gain_over_random_at_equal_trees(trained, mode):
    k = knng()
    X, net = trained
    n, kk = X.shape[0], 20
    Xd = torch.from_numpy(X).cuda()
    part = k.PART_RANDOM if mode == "embedding_random" else k.PART_FEATURES
    sample = synthetic.sample_ids(n, 2000, 5)
    T = 2
    r_rand = _recall(X, k.knng_build(Xd, kk, T, 256, 0, 21)[0], kk, sample)
    ids, dd = k.knng_build_learned(net, Xd, kk, T, 256, 0, 21, partitioner=part)
    r_lrn = _recall(X, ids, kk, sample)
    print(f"recall T=2, no propagation: random {r_rand:.4f}, learned ({mode}) {r_lrn:.4f}")
    ids = ids.cpu().numpy()
    assert np.all((ids >= -1) & (ids < n))
    assert r_lrn > r_rand, (r_lrn, r_rand)


def test_learned_embedding_build_matches_oracle_stagewise(trained):
    # the embedding trees are the random partition of the points z = f(x)
    # (the GPU's BF16 inference), the lists those of the rows x
    k = knng()
    X, net = trained
    X = np.ascontiguousarray(X[:8000])
    Xd = torch.from_numpy(X).cuda()
    Z = k.knng_mlp_forward(net, Xd).cpu().numpy()
    T, g, kk, seed = 3, 64, 10, 4
    gi, gd = k.knng_build_learned(net, Xd, kk, T, g, 1, seed)
    Xf = X.astype(np.float32)
    lists = np.empty((T, 8000, kk), dtype=np.int32)
    for t in range(T):
        perm, off = oracle.partition(Z, seed, t, g)
        np.testing.assert_array_equal(k.knng_partition(torch.from_numpy(Z).cuda(), T, g, seed)[t].cpu().numpy(),
                                      perm)
        lists[t], _ = oracle.leaf_knn(Xf, perm, off, kk)
    oi, od = oracle.merge(Xf, lists, kk)
    oi, od = oracle.propagate(Xf, oi, kk)
    gi = gi.cpu().numpy()
    assert np.mean(gi == oi) > 0.99
