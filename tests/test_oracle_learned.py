"""Pins of the oracle's learned-partitioner pieces (CPU): the per-level
feature splits (partition_features) and the feature order of each tree.

The learned partitioner is not in the paper; its split rule is the one the
library states for KNNG_PART_FEATURES: level l < C of tree t splits a node at
the median of feature pi_t(l) while that feature still varies inside the
node (range in the node > tau x range over all points), and at the median of
the node's random direction otherwise and past level C.
"""
import numpy as np

import oracle


def _leaf_sizes(m, g):
    # the floor/ceil halving of Sec. 3.1's recursive bisection
    if m <= g:
        return [m]
    return _leaf_sizes(m // 2, g) + _leaf_sizes(m - m // 2, g)


def _chunks(order, g):
    out, p = [], 0
    for s in _leaf_sizes(len(order), g):
        out.append(np.sort(order[p:p + s]))
        p += s
    return np.concatenate(out)


def test_feature_order_is_a_uniform_permutation():
    # Fisher-Yates draws every permutation equally often; Sattolo's variant
    # (j < i) or the naive shuffle (j over all C) would not
    C, trials = 4, 12000
    counts = {}
    for t in range(trials):
        p = tuple(oracle.feature_order(77, t, C))
        assert sorted(p) == list(range(C))
        counts[p] = counts.get(p, 0) + 1
    assert len(counts) == 24
    exp = trials / 24
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 60, chi2          # 23 degrees of freedom: p < 1e-4 above 52
    for i in range(16):
        assert sorted(oracle.feature_order(3, i, 16)) == list(range(16))


def test_increasing_features_reduce_the_split_to_sorting():
    # every feature strictly increasing in x0, depth <= C: each split is a
    # median split of x0, so the leaves are consecutive runs of the points
    # sorted by x0, sized by the halving rule, members by id
    rng = np.random.default_rng(1)
    n, d, C, g = 1000, 5, 16, 16
    X = rng.normal(size=(n, d)).astype(np.float32)
    X[:, 0] = rng.permutation(n).astype(np.float32)
    a = rng.uniform(0.5, 2.0, size=C).astype(np.float32)
    b = rng.uniform(-3, 3, size=C).astype(np.float32)
    Z = (X[:, :1] * a + b).astype(np.float32)
    for t in range(3):
        perm, off = oracle.partition_features(X, Z, 11, t, g)
        np.testing.assert_array_equal(perm, _chunks(np.argsort(X[:, 0], kind="stable"), g))
        np.testing.assert_array_equal(np.diff(off), _leaf_sizes(n, g))


def test_decreasing_features_split_in_descending_order():
    rng = np.random.default_rng(2)
    n, d, C, g = 700, 3, 16, 20
    X = rng.normal(size=(n, d)).astype(np.float32)
    X[:, 0] = rng.permutation(n).astype(np.float32)
    Z = np.repeat(-X[:, :1], C, axis=1).astype(np.float32)
    perm, _ = oracle.partition_features(X, Z, 5, 0, g)
    np.testing.assert_array_equal(perm, _chunks(np.argsort(-X[:, 0], kind="stable"), g))


def test_flat_features_fall_back_to_the_random_partition():
    rng = np.random.default_rng(3)
    n, d, C, g = 2000, 12, 16, 24
    X = np.rint(rng.normal(size=(n, d)) * 40).astype(np.float32)
    Z = np.full((n, C), 0.25, dtype=np.float32)
    for t in range(2):
        got = oracle.partition_features(X, Z, 9, t, g)
        want = oracle.partition(X, 9, t, g)
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])


def _level1_split_by(Z, f, members):
    # the first child of a node split at the median of feature f
    keys = sorted((float(Z[i, f]), int(i)) for i in members)
    return np.sort([i for _, i in keys[: len(members) // 2]])


def test_flatness_threshold_is_strict_and_scaled_by_the_global_range():
    # the root splits on feature pi(0) = x0 order; in the left child feature
    # pi(1) spans exactly tau x (its global range 1.0): not more than the bar,
    # so that node falls back to its random direction; nudging the span one
    # FP32 step above the bar makes it split on the feature
    n, d, C, g, seed, t = 64, 4, 16, 8, 21, 0
    rng = np.random.default_rng(4)
    order = oracle.feature_order(seed, t, C)
    f0, f1 = int(order[0]), int(order[1])
    X = rng.normal(size=(n, d)).astype(np.float32)
    x0 = np.arange(n, dtype=np.float32)
    left, right = np.arange(n // 2), np.arange(n // 2, n)
    bar = np.float32(oracle.LEARNED_TAU) * np.float32(1.0)

    def make(span_left):
        Z = np.zeros((n, C), dtype=np.float32)
        Z[:, f0] = x0
        # feature f1: the global range is 1.0 (set in the right child); in the
        # left child its values cover [0, span_left]
        vals = np.linspace(0.0, 1.0, n // 2, dtype=np.float32)
        Z[right, f1] = rng.permutation(vals)
        Z[left, f1] = rng.permutation(np.linspace(0.0, 1.0, n // 2).astype(np.float32) * span_left)
        Z[left[0], f1] = np.float32(span_left)
        Z[left[1], f1] = np.float32(0.0)
        return Z

    on_bar = make(bar)
    assert np.float32(on_bar[left, f1].max() - on_bar[left, f1].min()) == bar
    perm, off = oracle.partition_features(X, on_bar, seed, t, g)
    # right child: split on f1
    np.testing.assert_array_equal(np.sort(perm[n // 2: 3 * n // 4]), _level1_split_by(on_bar, f1, right))
    # left child: the random direction of node (level 1, v 0)
    a = oracle.direction(seed, t, 1, 0, d)
    proj = [(oracle.ord32(oracle.project(X[i], a)), int(i)) for i in left]
    want = np.sort([i for _, i in sorted(proj)[: n // 4]])
    np.testing.assert_array_equal(np.sort(perm[: n // 4]), want)
    above = make(np.nextafter(bar, np.float32(1.0)))
    perm2, _ = oracle.partition_features(X, above, seed, t, g)
    np.testing.assert_array_equal(np.sort(perm2[: n // 4]), _level1_split_by(above, f1, left))
    assert not np.array_equal(np.sort(perm2[: n // 4]), want)


def test_levels_past_the_features_use_random_directions():
    # C features and more than C levels.  With n = 2^18 every node of level l
    # is an aligned run of 2^(18-l) consecutive x0 ranks, and the feature of
    # level l is x0 mod 2^(18-l): increasing inside each such run and spanning
    # its whole global range there, so the first C levels sort by x0; deeper
    # nodes split along their random directions -- a leaf's members then need
    # not be consecutive in x0
    rng = np.random.default_rng(5)
    C, g, seed = 16, 2, 2
    n = 2 ** 18                 # 17 split levels at leaf size 2
    X = rng.normal(size=(n, 3)).astype(np.float32)
    r0 = rng.permutation(n)
    X[:, 0] = r0.astype(np.float32)
    Z = np.zeros((n, C), dtype=np.float32)
    for lvl, f in enumerate(oracle.feature_order(seed, 0, C)):
        Z[:, f] = (r0 % (2 ** (18 - lvl))).astype(np.float32)
    perm, off = oracle.partition_features(X, Z, seed, 0, g)
    assert sorted(perm.tolist()) == list(range(n))
    # after C levels the nodes are consecutive x0 runs: every node of level C
    # (or leaf above it) holds a run, whatever the deeper splits did
    rank = np.empty(n, dtype=np.int64)
    rank[np.argsort(X[:, 0], kind="stable")] = np.arange(n)

    def units(m, level, stop):
        if m <= g or level == stop:
            return [m]
        return units(m // 2, level + 1, stop) + units(m - m // 2, level + 1, stop)

    def runs(sizes):
        p, ok = 0, []
        for s in sizes:
            r = np.sort(rank[perm[p:p + s]])
            ok.append(r[-1] - r[0] == s - 1)
            p += s
        return np.array(ok)

    assert runs(units(n, 0, C)).all()
    # level C itself splits by a random direction, not by x0: many of its
    # children are not x0 runs
    deeper = runs(units(n, 0, C + 1))
    assert (~deeper).sum() > len(deeper) // 8
