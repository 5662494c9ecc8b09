"""FP64 oracle of the learned partitioner's network and training loss.

TEST INFRASTRUCTURE (see oracle/__init__.py): the plain NumPy statement of
what the CUDA training kernels compute, used to check their gradients.

The paper has no learned partitioner; this is the reading used by the
library.  Network (FP32 weights on the GPU):

    A = X W1^T + b1          (N x H)
    Hh = GELU(A)             GELU(a) = a/2 (1 + erf(a / sqrt 2))
    Z = tanh(Hh W2^T + b2)   (N x C)

The outputs are bounded so that no output can lower the loss by inflating
its spread with a few outliers (tanh is monotone, so splits at a median are
unaffected by it).

Loss on a batch of B graph edges (i_b, j_b): rows 0..B-1 of X are the first
endpoints, rows B..2B-1 the second ones (N = 2B).  With the batch mean mu_c
and variance V_c of every output c over the N rows,

    L_pair = sum_c  mean_b (Z[b,c] - Z[B+b,c])^2 / (V_c + eps)
    S      = (Z - mu) / sqrt(V + eps),    K = S^T S / N
    L_dec  = sum_{c != c'} K[c,c']^2
    L_spr  = sum_c (1 - V_c)^2
    L      = L_pair + lam * L_dec + mu_s * L_spr

Neighbours should fall on the same side of a median split: each output
should vary little along graph edges relative to its spread (L_pair), the
outputs should carry different information (L_dec), and no output may
collapse to a constant (L_spr: with outputs in (-1, 1) the spread is largest
for balanced +-1 values).
"""
from __future__ import annotations

import math

import numpy as np

from . import philox4x32_10

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def _erf(x):
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def gelu(a):
    return 0.5 * a * (1.0 + _erf(a / SQRT2))


def gelu_grad(a):
    return 0.5 * (1.0 + _erf(a / SQRT2)) + a * INV_SQRT_2PI * np.exp(-0.5 * a * a)


def forward(X, W1, b1, W2, b2):
    X = np.asarray(X, dtype=np.float64)
    A = X @ np.asarray(W1, np.float64).T + np.asarray(b1, np.float64)
    Hh = gelu(A)
    Z = np.tanh(Hh @ np.asarray(W2, np.float64).T + np.asarray(b2, np.float64))
    return A, Hh, Z


def loss_from_z(Z, lam, eps, mu_s=1.0):
    """Loss and dL/dZ (both FP64) for the pair batch Z (2B x C)."""
    Z = np.asarray(Z, dtype=np.float64)
    N, C = Z.shape
    B = N // 2
    mu = Z.mean(axis=0)
    Zc = Z - mu
    V = (Zc * Zc).mean(axis=0)
    D = Z[:B] - Z[B:]
    P = (D * D).mean(axis=0)
    L_pair = float(np.sum(P / (V + eps)))
    sig = np.sqrt(V + eps)
    S = Zc / sig
    K = S.T @ S / N
    off = K - np.diag(np.diag(K))
    L_dec = float(np.sum(off * off))
    L_spr = float(np.sum((1.0 - V) ** 2))
    L = L_pair + lam * L_dec + mu_s * L_spr
    # gradient
    dZ = np.zeros_like(Z)
    dP = 1.0 / (V + eps)                      # dL/dP_c
    dV = -P / (V + eps) ** 2 - 2.0 * mu_s * (1.0 - V)   # dL/dV_c (pair and spread terms)
    dZ[:B] += dP * (2.0 / B) * D
    dZ[B:] -= dP * (2.0 / B) * D
    dZ += dV * (2.0 / N) * Zc
    G = 2.0 * off * lam                       # dL/dK (symmetric, zero diagonal)
    dS = (2.0 / N) * S @ G                    # K = S^T S / N
    # through S = (Z - mu) / sqrt(V + eps), per column
    m1 = dS.mean(axis=0)
    m2 = (dS * S).mean(axis=0)
    dZ += (dS - m1 - S * m2) / sig
    return L, dZ


def loss_and_grads(X, W1, b1, W2, b2, lam=0.05, eps=1e-4, mu_s=1.0):
    """Loss and gradients with respect to (W1, b1, W2, b2), FP64."""
    X = np.asarray(X, dtype=np.float64)
    A, Hh, Z = forward(X, W1, b1, W2, b2)
    L, dZ = loss_from_z(Z, lam, eps, mu_s)
    dZ = dZ * (1.0 - Z * Z)   # through the output tanh
    dW2 = dZ.T @ Hh
    db2 = dZ.sum(axis=0)
    dH = dZ @ np.asarray(W2, np.float64)
    dA = dH * gelu_grad(A)
    dW1 = dA.T @ X
    db1 = dA.sum(axis=0)
    return L, (dW1, db1, dW2, db2)


# --------------------------------------------------------------- training --
# The training loop draws each batch from the graph with Philox4x32-10 and
# takes one Adam step (Kingma and Ba, "Adam: a method for stochastic
# optimization", ICLR 2015, Algorithm 1) per batch.

BATCH_TAG = 0x4C4E4E42


def sample_batch(X, ids, B: int, seed: int, step: int) -> np.ndarray:
    """The FP32 pair rows [2B, d] of training step `step`: edge b takes point
    i = (w0 * 2^32 + w1) mod n and the first valid entry of i's list at slots
    ((w2 + t) mod 2^32) mod k, t = 0, 1, ... (i itself if the list is empty),
    where
    (w0..w3) = Philox4x32-10(counter (b, step, BATCH_TAG, 0), key seed).
    Row b is x_i, row B + b is x_j."""
    X = np.asarray(X)
    X = X.astype(np.float32) if X.dtype != np.float32 else X
    ids = np.asarray(ids)
    n, k = ids.shape
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    out = np.empty((2 * B, X.shape[1]), dtype=np.float32)
    for b in range(B):
        w = [int(x) for x in philox4x32_10((b, step, BATCH_TAG, 0), key)]
        i = ((w[0] << 32) | w[1]) % n
        j = -1
        for t in range(k):
            j = int(ids[i, ((w[2] + t) & 0xFFFFFFFF) % k])
            if j >= 0:
                break
        if j < 0 or j >= n:
            j = i
        out[b] = X[i]
        out[B + b] = X[j]
    return out


def adam_step(w, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """Step t (1-based) of Adam, FP64: returns the new (w, m, v)."""
    w, g, m, v = (np.asarray(a, dtype=np.float64) for a in (w, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v
