"""First-order propagation (Sec. 3.2) on input graphs that did not come from
the merge: rows in arbitrary order and rows with empty slots.  A round's
result depends only on the sets of listed neighbours (the k best by
(distance, id) of a point's list and its neighbours' lists), so it must
equal the oracle's exactly on integer-valued rows, whatever the order of
the input rows' entries.
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


def _merged(X, k, T, g, seed):
    Xd = dev(X)
    perm = knng().knng_partition(Xd, T, g, seed)
    li, ld = knng().knng_leaf_knn(Xd, T, g, perm, k)
    mi, md = knng().knng_merge(li, ld)
    return Xd, host(mi), host(md)


@pytest.mark.parametrize("k", [10, 20, 32])
def test_unordered_and_partial_rows(k):
    X = synthetic.sift_like(8000, 64, centers=40, seed=k)
    Xd, mi, md = _merged(X, k, 3, max(2 * k + 2, 64), 5)
    rng = np.random.default_rng(k)
    n = X.shape[0]
    ids, dists = mi.copy(), md.copy()
    # a third of the rows shuffled, a sixth with empty slots (anywhere)
    for p in rng.choice(n, n // 3, replace=False):
        o = rng.permutation(k)
        ids[p], dists[p] = ids[p][o], dists[p][o]
    for p in rng.choice(n, n // 6, replace=False):
        drop = rng.random(k) < 0.3
        ids[p][drop] = -1
        dists[p][drop] = np.inf
    gi, gd = knng().knng_propagate(Xd, dev(ids), dev(dists), 1)
    oi, od = oracle.propagate(X, ids, k)
    np.testing.assert_array_equal(host(gi), oi)
    np.testing.assert_array_equal(host(gd), od)
    # a second round on the GPU's own output (ordered, full rows)
    hi, hd = knng().knng_propagate(Xd, gi, gd, 1)
    oi2, od2 = oracle.propagate(X, oi, k)
    np.testing.assert_array_equal(host(hi), oi2)
    np.testing.assert_array_equal(host(hd), od2)
