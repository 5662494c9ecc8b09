"""FP64 oracle of the random principal directions (Sec. 3.4, "Random
division": the split direction of a node is the principal direction of
points sampled at random from it, computed by the Lanczos algorithm).

TEST INFRASTRUCTURE (see oracle/__init__.py): only the tests, the smoke
check and the benchmark's CPU legs may use it.  NumPy, FP64.

The paper gives neither the sample size nor the number of Lanczos steps;
the readings used here (the kernel takes the same ones):

* sample: a node of m points (ids ascending) with m <= s_cap uses all of
  them; otherwise s_cap points M[w_r mod m], r = 0 .. s_cap - 1, where w_r is
  word r mod 4 of Philox4x32-10 with counter (t, level | 2^30, v, r // 4) and
  key = seed (with replacement).  s_cap = clamp(floor(40960 / d), 8, 128).
* covariance of the sample, C = A^T A / s with A the centred rows.
* the textbook Lanczos recurrence, alpha_j = v_j . C v_j and
  w = C v_j - alpha_j v_j - beta_{j-1} v_{j-1}, with full reorthogonalisation
  (w is orthogonalised against every earlier basis vector by classical
  Gram-Schmidt, applied twice: a second pass restores orthogonality to
  working precision), from the node's random direction (the one the random
  partitioner would use, normalised), at most q = min(8, d) steps, stopping
  once beta_j <= 1e-4 * max_i alpha_i.
* the Ritz vector of the largest eigenvalue of the tridiagonal matrix,
  normalised, with its largest-magnitude entry made positive (ties: the
  lowest index).
"""
from __future__ import annotations

import numpy as np

from . import direction, philox4x32_10

STEPS = 8
LEVEL_TAG = 1 << 30


def sample_cap(d: int) -> int:
    return int(min(128, max(8, 40960 // d)))


def sample_rows(members, seed: int, t: int, level: int, v: int, d: int) -> np.ndarray:
    """The sampled member ids of node (t, level, v); members ascending."""
    members = np.asarray(members)
    m = members.shape[0]
    cap = sample_cap(d)
    if m <= cap:
        return members.copy()
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    idx = np.empty(cap, dtype=np.int64)
    for r in range(cap):
        if r % 4 == 0:
            w = philox4x32_10((t, level | LEVEL_TAG, v, r // 4), key)
        idx[r] = int(w[r % 4]) % m
    return members[idx]


def lanczos_top(C_mul, v0: np.ndarray, steps: int, with_value: bool = False):
    """Top Ritz vector of the symmetric operator C_mul after at most
    `steps` Lanczos steps with full reorthogonalisation, from v0 (and its
    Ritz value when with_value)."""
    d = v0.shape[0]
    V = np.zeros((steps + 1, d))
    V[0] = v0 / np.linalg.norm(v0)
    alpha, beta = [], []
    amax = 0.0
    for j in range(steps):
        w = C_mul(V[j])
        a = float(V[j] @ w)
        alpha.append(a)
        amax = max(amax, a)
        # three-term recurrence
        w = w - a * V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        # full reorthogonalisation: classical Gram-Schmidt, twice
        for _ in range(2):
            w = w - V[:j + 1].T @ (V[:j + 1] @ w)
        b = float(np.linalg.norm(w))
        if j == steps - 1 or b <= 1e-4 * amax:
            break
        beta.append(b)
        V[j + 1] = w / b
    q = len(alpha)
    Tm = np.diag(alpha)
    for i, b in enumerate(beta[:q - 1]):
        Tm[i, i + 1] = Tm[i + 1, i] = b
    evals, evecs = np.linalg.eigh(Tm)
    y = evecs[:, -1]
    a = V[:q].T @ y
    a /= np.linalg.norm(a)
    i = int(np.argmax(np.abs(a)))
    if a[i] < 0:
        a = -a
    return (a, float(evals[-1])) if with_value else a


def sample_covariance(X, members, seed: int, t: int, level: int, v: int) -> np.ndarray:
    """C = A^T A / s of the node's sampled rows A, centred (FP64)."""
    X = np.asarray(X)
    rows = sample_rows(members, seed, t, level, v, X.shape[1])
    A = X[rows].astype(np.float64)
    A = A - A.mean(axis=0)
    return A.T @ A / A.shape[0]


def principal_direction(X, members, seed: int, t: int, level: int, v: int, with_value: bool = False):
    """Split direction of node (t, level, v) whose members (ascending ids)
    are given: the principal direction of the sampled, centred rows (and its
    Ritz value, the variance along it, when with_value)."""
    X = np.asarray(X)
    d = X.shape[1]
    rows = sample_rows(members, seed, t, level, v, d)
    A = X[rows].astype(np.float64)
    A = A - A.mean(axis=0)
    s = A.shape[0]
    v0 = direction(seed, t, level, v, d).astype(np.float64)
    return lanczos_top(lambda x: A.T @ (A @ x) / s, v0, min(STEPS, d), with_value)
