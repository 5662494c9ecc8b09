"""Seeded synthetic point sets shaped like the paper's workloads.

The paper measures on 1M SIFT-128 and 1M GIST descriptors (Sec. 4); those sets
are not available here, so these Gaussian mixtures stand in for them.  This
module holds only input generation (NumPy ``Generator(PCG64(seed))``); none
of the method's arithmetic is here, and both the CUDA path and the CPU oracle
are fed from it.

* ``sift_like``  -- centres uniform in [0, 255]^d, per-dimension N(0, std^2)
  noise, rounded and clipped to the integers 0..255 (float32 storage).
* ``gist_like``  -- centres uniform in [0, 1]^d, N(0, std^2) noise, clipped
  to [0, 1], every row L2-normalised (float32).
* ``sphere_f16`` -- centres = normalised N(0, I), N(0, std^2) noise, rows
  normalised, stored as float16.
* ``batched_sets`` -- many independent float32 mixtures with log-uniform n.

Every point draws its centre uniformly at random.
"""
from __future__ import annotations

import numpy as np

_CHUNK = 1 << 17


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sift_like(n: int, d: int = 128, centers: int = 1024, std: float = 20.0,
              seed: int = 0) -> np.ndarray:
    rng = _rng(seed)
    C = rng.uniform(0.0, 255.0, size=(centers, d))
    lab = rng.integers(0, centers, size=n)
    X = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        v = C[lab[s:e]] + rng.normal(0.0, std, size=(e - s, d))
        X[s:e] = np.clip(np.rint(v), 0.0, 255.0)
    return X


def gist_like(n: int, d: int = 960, centers: int = 256, std: float = 0.1,
              seed: int = 0) -> np.ndarray:
    rng = _rng(seed)
    C = rng.uniform(0.0, 1.0, size=(centers, d))
    lab = rng.integers(0, centers, size=n)
    X = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        v = np.clip(C[lab[s:e]] + rng.normal(0.0, std, size=(e - s, d)), 0.0, 1.0)
        nrm = np.linalg.norm(v, axis=1, keepdims=True)
        nrm[nrm == 0.0] = 1.0
        X[s:e] = v / nrm
    return X


def sphere_f16(n: int, d: int = 96, centers: int = 4096, std: float = 0.05,
               seed: int = 0) -> np.ndarray:
    rng = _rng(seed)
    C = rng.normal(0.0, 1.0, size=(centers, d))
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    lab = rng.integers(0, centers, size=n)
    X = np.empty((n, d), dtype=np.float16)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        v = C[lab[s:e]] + rng.normal(0.0, std, size=(e - s, d))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        X[s:e] = v.astype(np.float16)
    return X


def gaussian_mixture(n: int, d: int, centers: int, std: float = 0.1,
                     seed: int = 0) -> np.ndarray:
    """Centres N(0, I), N(0, std^2) noise, float32 (the batched-set law)."""
    rng = _rng(seed)
    C = rng.normal(0.0, 1.0, size=(centers, d))
    lab = rng.integers(0, centers, size=n)
    X = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        X[s:e] = C[lab[s:e]] + rng.normal(0.0, std, size=(e - s, d))
    return X


def batched_sets(count: int = 256, n_lo: int = 2000, n_hi: int = 200000,
                 dims=(64, 128, 256), c_lo: int = 16, c_hi: int = 256,
                 std: float = 0.1, seed: int = 0):
    """``count`` independent mixtures: n log-uniform in [n_lo, n_hi], d drawn
    from ``dims``, centre count uniform in [c_lo, c_hi]."""
    rng = _rng(seed)
    out = []
    for s in range(count):
        n = int(round(float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))))
        d = int(rng.choice(np.asarray(dims)))
        c = int(rng.integers(c_lo, c_hi + 1))
        out.append(gaussian_mixture(n, d, c, std, seed=seed * 1000003 + s + 1))
    return out


def sample_ids(n: int, count: int, seed: int) -> np.ndarray:
    """Sorted distinct point ids for a recall sample."""
    rng = _rng(seed)
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False)).astype(np.int32)
