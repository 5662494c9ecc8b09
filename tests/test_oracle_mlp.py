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
