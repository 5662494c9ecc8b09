"""Learned partitioner on the GPU, through the C ABI: training gradients
against the FP64 oracle, BF16 inference against the FP64 forward pass, the
training loop, persistence, and what the trained network gains over random
directions at an equal number of trees."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1307_7852_gb300 import synthetic
from validity import check_build_stagewise

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


@pytest.mark.parametrize("mode", ["embedding", "features"])
def test_learned_build_matches_oracle_stagewise(trained, mode):
    # the learned build through its stages: the partition of the GPU's network
    # outputs z (random trees on z, or per-level feature splits) bit-exact,
    # then the lists of the rows x, every row checked in full
    k = knng()
    X, net = trained
    X = np.ascontiguousarray(X[:8000])
    Xd = torch.from_numpy(X).cuda()
    T, g, kk, seed = 3, 64, 10, 4
    part = k.PART_RANDOM if mode == "embedding" else k.PART_FEATURES
    gi, gd = k.knng_build_learned(net, Xd, kk, T, g, 1, seed, partitioner=part)
    check_build_stagewise(k, torch, X, kk, T, g, 1, seed, gi.cpu().numpy(), gd.cpu().numpy(), net=net,
                          learned=mode)


def test_feature_partition_bit_exact(trained):
    # the per-level learned-feature partition replayed by the oracle on the
    # GPU's own network outputs (BF16 inference) is bit-exact
    k = knng()
    X, net = trained
    T, g, seed = 3, 48, 17
    perm, Z = k.knng_partition_learned(net, torch.from_numpy(X).cuda(), T, g, seed, with_z=True)
    perm, Z = perm.cpu().numpy(), Z.cpu().numpy()
    for t in range(T):
        np.testing.assert_array_equal(perm[t], oracle.partition_features(X, Z, seed, t, g)[0])


def test_feature_partition_flat_outputs_and_deep_trees():
    # outputs 0..7 constant (zero output weights): those levels fall back to
    # random directions of x; 140,000 points at leaf size 2 need 17 levels,
    # one more than the 16 outputs
    k = knng()
    net = k.Mlp(96, 64, 16, seed=8)
    W1, b1, W2, b2 = net.get_params()
    W2 = W2.copy()
    W2[:8] = 0.0
    b2 = b2.copy()
    b2[:8] = np.linspace(-0.5, 0.5, 8, dtype=np.float32)
    net.set_params(W1, b1, W2, b2)
    X = synthetic.sphere_f16(140000, 96, centers=64, seed=12)
    T, g, seed = 2, 2, 23
    perm, Z = k.knng_partition_learned(net, torch.from_numpy(X).cuda(), T, g, seed, with_z=True)
    perm, Z = perm.cpu().numpy(), Z.cpu().numpy()
    assert np.all(Z[:, :8] == Z[0, :8])
    for t in range(T):
        np.testing.assert_array_equal(perm[t], oracle.partition_features(X, Z, seed, t, g)[0])


def test_adam_step_matches_fp64_oracle():
    # one training step from a given Adam state: the batch the GPU draws is
    # the oracle's sampler's (Philox), its gradient the GPU's own (checked
    # against FP64 above), and the update must be the FP64 Adam step of it
    k = knng()
    rng = np.random.default_rng(4)
    net = k.Mlp(32, 64, 16, seed=6)
    n, kk, B, lr, seed = 3000, 8, 256, 3e-3, 41
    X = rng.normal(size=(n, 32)).astype(np.float32)
    ids = rng.integers(0, n, size=(n, kk)).astype(np.int32)
    ids[5, :] = -1
    P = net.param_count()
    w0 = np.concatenate([a.ravel() for a in net.get_params()]).astype(np.float32)
    m0 = (rng.normal(size=P) * 1e-2).astype(np.float32)
    v0 = (rng.uniform(0, 1e-4, size=P)).astype(np.float32)
    net.set_adam_state(m0, v0, 5)
    Xp = omlp.sample_batch(X, ids, B, seed, 0)
    _, g = net.loss_grad(torch.from_numpy(Xp).cuda())
    g = g.cpu().numpy()
    Xd, idd = torch.from_numpy(X).cuda(), torch.from_numpy(ids).cuda()
    net.train(Xd, idd, 1, batch_edges=B, lr=lr, seed=seed)
    w1 = np.concatenate([a.ravel() for a in net.get_params()])
    m1, v1, t1 = net.get_adam_state()
    assert t1 == 6
    # the kernel's constants are the FP32 numbers nearest 0.9, 0.999 and 1e-8;
    # the oracle takes those exact values, so what remains is FP32 rounding
    b1, b2, eps = (float(np.float32(v)) for v in (0.9, 0.999, 1e-8))
    ow, om, ov = omlp.adam_step(w0, g, m0, v0, 6, lr, b1=b1, b2=b2, eps=eps)
    g64 = g.astype(np.float64)
    # m = b1 m + (1 - b1) g may cancel: a few units of 2^-24 of its terms
    tol_m = 2.0 ** -21 * (np.abs(b1 * m0) + np.abs((1 - b1) * g64))
    assert np.all(np.abs(m1 - om) <= tol_m), np.max(np.abs(m1 - om) / tol_m)
    np.testing.assert_allclose(v1, ov, rtol=1e-6, atol=1e-30)
    # the step lr * mhat / (sqrt(vhat) + eps) inherits m's error; w's own
    # rounding adds a unit in its last place
    c1, c2 = 1 - b1 ** 6, 1 - b2 ** 6
    step = np.abs(ow - w0)
    tol_w = (2 * np.spacing(np.abs(w0).astype(np.float32)).astype(np.float64)
             + lr * (tol_m / c1) / (np.sqrt(ov / c2) + eps) + 1e-5 * step)
    assert np.all(np.abs(w1 - ow) <= tol_w), np.max(np.abs(w1 - ow) / tol_w)
    assert np.median(step) > 1e-4      # the step is not vacuous
