"""Pins of the oracle's random principal directions (Sec. 3.4) and of the
partition replay with given directions (CPU)."""
import numpy as np

import oracle
from oracle import pca
from paper_1307_7852_gb300 import synthetic


def test_points_on_a_line_give_the_line():
    rng = np.random.default_rng(1)
    u = rng.normal(size=40)
    u /= np.linalg.norm(u)
    X = (rng.normal(size=(500, 1)) * 10.0 * u + 0.01 * rng.normal(size=(500, 40))).astype(np.float32)
    a = pca.principal_direction(X, np.arange(500), 3, 0, 0, 0)
    assert abs(a @ u) > 0.9999
    assert abs(np.linalg.norm(a) - 1.0) < 1e-12


def test_full_krylov_space_is_the_exact_top_eigenvector():
    # d <= 8: the Lanczos steps span the whole space, so the Ritz vector is
    # the top eigenvector of the sample covariance (library eigensolver)
    rng = np.random.default_rng(2)
    X = (rng.normal(size=(90, 6)) * np.array([3.0, 1.0, 0.5, 2.0, 0.2, 1.5])).astype(np.float32)
    members = np.arange(90)
    a = pca.principal_direction(X, members, 5, 1, 2, 3)
    rows = pca.sample_rows(members, 5, 1, 2, 3, 6)
    A = X[rows].astype(np.float64)
    A -= A.mean(0)
    w, V = np.linalg.eigh(A.T @ A / A.shape[0])
    top = V[:, -1]
    assert abs(abs(a @ top) - 1.0) < 1e-10
    i = int(np.argmax(np.abs(a)))
    assert a[i] > 0


def test_anisotropic_cloud_gives_its_long_axis():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(64, 64)))
    sd = np.ones(64)
    sd[0] = 6.0
    X = ((rng.normal(size=(20000, 64)) * sd) @ Q.T).astype(np.float32)
    a = pca.principal_direction(X, np.arange(20000), 9, 0, 0, 0)   # 128 sampled rows
    assert abs(a @ Q[:, 0]) > 0.98


def test_sample_rule():
    members = np.arange(1000, 1100)
    np.testing.assert_array_equal(pca.sample_rows(members, 1, 0, 0, 0, 128), members)   # 100 <= 128
    big = np.arange(5000) * 3
    r = pca.sample_rows(big, 1, 2, 3, 4, 128)
    assert r.shape == (128,) and np.all(np.isin(r, big)) and len(np.unique(r)) > 100
    np.testing.assert_array_equal(r, pca.sample_rows(big, 1, 2, 3, 4, 128))
    assert pca.sample_cap(960) == 42 and pca.sample_cap(128) == 128 and pca.sample_cap(4096) == 10


def test_replay_with_the_random_directions_is_the_random_partition():
    X = synthetic.sift_like(3000, 24, centers=8, seed=4)
    g, seed, t = 40, 7, 1
    nodes = oracle.split_nodes(3000, g)
    depth = max(l for l, *_ in nodes) + 1
    dirs = np.zeros((2 ** depth - 1, 24), dtype=np.float32)
    for (l, v, off, m) in nodes:
        dirs[2 ** l - 1 + v] = oracle.direction(seed, t, l, v, 24)
    p1, o1 = oracle.partition_with_dirs(X, dirs, g)
    p0, o0 = oracle.partition(X, seed, t, g)
    np.testing.assert_array_equal(p1, p0)
    np.testing.assert_array_equal(o1, o0)


def test_split_node_table_matches_the_leaf_layout():
    n, g = 10000, 64
    nodes = oracle.split_nodes(n, g)
    assert nodes[0] == (0, 0, 0, n)
    # leaves = children of split nodes that are not split themselves
    split = {(l, v) for l, v, _, _ in nodes}
    leaves = []
    for l, v, off, m in nodes:
        for c, (o, mm) in enumerate(((off, m // 2), (off + m // 2, m - m // 2))):
            if (l + 1, 2 * v + c) not in split:
                leaves.append((o, mm))
    leaves.sort()
    off = oracle.partition(synthetic.sift_like(n, 8, centers=4, seed=1), 1, 0, g)[1]
    np.testing.assert_array_equal([o for o, _ in leaves] + [n], off)
