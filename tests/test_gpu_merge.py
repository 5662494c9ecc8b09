"""Combination of the T base graphs (Sec. 3.1) on the GPU, through the C ABI,
at the shapes the end-to-end tests do not reach: one tree and up to 32, k up
to 64, a number of points that leaves a ragged last batch; and hand-made
rows in which a neighbour appears in several trees with equal or different
distances, next to p itself and empty slots.

Leaf lists of integer-valued rows carry exact distances, so the merge must
equal the oracle's exactly.  The hand-made rows follow the entry point's
own rule: the union of the rows, each ordered by (distance, id), keeping the
first (smallest) entry of every id other than p, the k best.
"""
import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def knng():
    import paper_1307_7852_gb300 as k
    return k


def dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("T,k", [(1, 20), (8, 20), (9, 10), (16, 33), (17, 20), (32, 8), (8, 64), (3, 64)])
def test_merge_shapes_integer_exact(T, k):
    n = 3001
    X = synthetic.sift_like(n, 32, centers=16, seed=100 * T + k)
    g = max(2 * k + 2, 64)
    Xd = dev(X)
    perm = knng().knng_partition(Xd, T, g, 5)
    li, ld = knng().knng_leaf_knn(Xd, T, g, perm, k)
    mi, md = knng().knng_merge(li, ld)
    oi, od = oracle.merge(X, host(li), k)
    np.testing.assert_array_equal(host(mi), oi)
    np.testing.assert_array_equal(host(md), od)


def _merge_rule(ids, dists, k):
    T, n, kin = ids.shape
    out_i = np.full((n, k), -1, np.int32)
    out_d = np.full((n, k), np.inf, np.float32)
    for p in range(n):
        cand = []
        for t in range(T):
            for h in range(kin):
                if ids[t, p, h] < 0:
                    break
                cand.append((float(dists[t, p, h]), int(ids[t, p, h])))
        cand.sort()
        seen, r = set(), 0
        for dd, i in cand:
            if i == p or i in seen:
                continue
            seen.add(i)
            out_i[p, r], out_d[p, r] = i, dd
            r += 1
            if r == k:
                break
    return out_i, out_d


@pytest.mark.parametrize("T,k", [(6, 12), (12, 5), (2, 40)])
def test_merge_repeated_neighbours(T, k):
    rng = np.random.default_rng(T * 7 + k)
    n = 1003
    ids = np.full((T, n, k), -1, np.int32)
    dists = np.full((T, n, k), np.inf, np.float32)
    # a per-point pool of ids with a base distance each, so that trees share
    # neighbours; a tree sometimes reports a shared one at another distance
    for p in range(n):
        pool = np.unique((p + rng.integers(-25, 26, size=3 * k)) % n)
        base = rng.integers(0, 30, size=pool.size).astype(np.float32)
        for t in range(T):
            m = int(rng.integers(0, k + 1))
            pick = rng.choice(pool.size, size=min(m, pool.size), replace=False)
            dd = base[pick].copy()
            moved = rng.random(pick.size) < 0.2
            dd[moved] += rng.integers(1, 5, size=int(moved.sum())).astype(np.float32)
            row = sorted(zip(dd.tolist(), pool[pick].tolist()))
            for h, (dv, i) in enumerate(row):
                ids[t, p, h] = i
                dists[t, p, h] = dv
    mi, md = knng().knng_merge(dev(ids), dev(dists))
    ri, rd = _merge_rule(ids, dists, k)
    np.testing.assert_array_equal(host(mi), ri)
    np.testing.assert_array_equal(host(md), rd)
