"""Pins of the FP64 network/loss oracle of the learned partitioner: gradients
against central finite differences, GELU against its closed-form limits."""
import math

import numpy as np

from oracle import mlp


def _tiny(seed=0, d=5, H=7, C=3, B=6):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(2 * B, d))
    W1 = rng.normal(size=(H, d)) * 0.7
    b1 = rng.normal(size=H) * 0.2
    W2 = rng.normal(size=(C, H)) * 0.7
    b2 = rng.normal(size=C) * 0.2
    return X, [W1, b1, W2, b2]


def test_gelu_closed_forms():
    a = np.array([-30.0, -1.0, 0.0, 1.0, 30.0])
    g = mlp.gelu(a)
    assert g[0] == 0.0 or abs(g[0]) < 1e-100
    assert g[2] == 0.0 and abs(g[4] - 30.0) < 1e-12
    # GELU(1) = Phi(1) = (1 + erf(1/sqrt 2))/2 = 0.841344746...
    assert abs(g[3] - 0.8413447460685429) < 1e-15
    assert abs(g[3] - g[1] - 1.0) < 1e-15  # gelu(a) - gelu(-a) = a
    h = 1e-6
    fd = (mlp.gelu(a + h) - mlp.gelu(a - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(a), fd, rtol=1e-7, atol=1e-9)


def test_gradients_match_finite_differences():
    for seed in range(3):
        X, P = _tiny(seed)
        lam, eps = 0.3, 1e-3
        L, grads = mlp.loss_and_grads(X, *P, lam=lam, eps=eps)
        h = 1e-6
        for pi, (p, g) in enumerate(zip(P, grads)):
            flat = p.reshape(-1)
            gf = g.reshape(-1)
            for idx in range(flat.size):
                old = flat[idx]
                flat[idx] = old + h
                Lp, _ = mlp.loss_and_grads(X, *P, lam=lam, eps=eps)
                flat[idx] = old - h
                Lm, _ = mlp.loss_and_grads(X, *P, lam=lam, eps=eps)
                flat[idx] = old
                fd = (Lp - Lm) / (2 * h)
                assert abs(fd - gf[idx]) <= 1e-6 * max(1.0, abs(fd)), (pi, idx, fd, gf[idx])


def test_loss_terms_special_cases():
    # identical endpoints: the pair term vanishes
    rng = np.random.default_rng(4)
    Zh = rng.normal(size=(5, 3))
    Z = np.concatenate([Zh, Zh])
    L, _ = mlp.loss_from_z(Z, 0.0, 1e-12, 0.0)
    assert abs(L) < 1e-12
    # balanced, uncorrelated +-1 outputs shared by both endpoints: every term
    # vanishes (pair 0, correlation 0, spread V = 1)
    Z = np.array([[1.0, 1.0], [-1.0, 1.0], [1.0, -1.0], [-1.0, -1.0]] * 2)
    L, _ = mlp.loss_from_z(np.concatenate([Z, Z]), 1.0, 0.0, 1.0)
    assert abs(L) < 1e-12
    Zc = np.array([[1.0, 1.0], [-1.0, -1.0]] * 2)  # perfectly correlated columns
    L, _ = mlp.loss_from_z(np.concatenate([Zc, Zc]), 1.0, 0.0, 0.0)
    assert abs(L - 2.0) < 1e-12
    # collapse to a constant costs the spread term: C * mu_s
    L, _ = mlp.loss_from_z(np.full((8, 3), 0.3), 0.0, 1e-4, 2.0)
    assert abs(L - 6.0) < 1e-12


# ------------------------------------------------------------ training --
def test_adam_first_step_is_a_sign_step():
    # from zero moments the bias corrections make the first step
    # lr * g / (|g| + eps): a step of lr against the sign of the gradient
    rng = np.random.default_rng(0)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    g[3] = 0.0
    w1, m1, v1 = mlp.adam_step(w, g, np.zeros(50), np.zeros(50), 1, 0.01)
    np.testing.assert_allclose(w1, w - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)


def test_adam_constant_gradient_moves_at_the_learning_rate():
    # a constant gradient g: the bias-corrected moments equal g and g^2 at
    # every step, so each step moves every weight by lr * g / (|g| + eps)
    rng = np.random.default_rng(1)
    w0 = rng.normal(size=20)
    g = rng.normal(size=20)
    w, m, v = w0, np.zeros(20), np.zeros(20)
    for t in range(1, 8):
        w, m, v = mlp.adam_step(w, g, m, v, t, 3e-3)
    np.testing.assert_allclose(w, w0 - 7 * 3e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_batch_sampler_draws_graph_edges():
    rng = np.random.default_rng(2)
    n, k, d = 300, 5, 7
    X = rng.normal(size=(n, d)).astype(np.float32)
    ids = rng.integers(0, n, size=(n, k)).astype(np.int32)
    ids[7] = -1                       # an empty list: the edge is (i, i)
    P = mlp.sample_batch(X, ids, 400, 9, 3)
    rowid = {X[i].tobytes(): i for i in range(n)}
    hits = np.zeros(n)
    for b in range(400):
        i, j = rowid[P[b].tobytes()], rowid[P[400 + b].tobytes()]
        hits[i] += 1
        assert (j in ids[i]) or (i == 7 and j == 7)
    assert (hits > 0).sum() > 200     # points drawn across the whole set
    np.testing.assert_array_equal(P, mlp.sample_batch(X, ids, 400, 9, 3))
    assert not np.array_equal(P, mlp.sample_batch(X, ids, 400, 9, 4))
