"""The complete row checks of tests/validity.py on CPU: the oracle's own
lists pass, and each kind of mistake planted into a copy of them fails."""
import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic
from validity import check_quant_leaf, check_rows, merge_candidates, propagation_candidates


@pytest.fixture(scope="module")
def quant_case():
    X = synthetic.gist_like(1500, 48, centers=6, seed=3)
    g, k, kp = 64, 6, 12
    perm, off = oracle.partition(X, 5, 0, g)
    oi, od = oracle.leaf_knn_quant(X, perm, off, k, kp, oracle.PREC_BF16)
    return X, perm, off, oi, od, k, kp


def test_quant_leaf_accepts_the_oracle(quant_case):
    X, perm, off, oi, od, k, kp = quant_case
    check_quant_leaf(X, perm, off, oi, od, k, kp, oracle.PREC_BF16)


def _other_member(perm, off, p, row):
    L = np.searchsorted(off, np.nonzero(perm == p)[0][0], side="right") - 1
    mem = perm[off[L]:off[L + 1]]
    for c in mem[::-1]:
        if c != p and c not in row:
            return int(c)
    raise AssertionError


@pytest.mark.parametrize("mistake", ["far_member", "other_leaf", "distance", "duplicate", "order", "self"])
def test_quant_leaf_rejects_planted_mistakes(quant_case, mistake):
    X, perm, off, oi, od, k, kp = quant_case
    gi, gd = oi.copy(), od.copy()
    p = 77
    if mistake == "far_member":
        # a leaf member far outside the k' candidates replaces the k-th
        c = _other_member(perm, off, p, gi[p])
        gi[p, -1] = c
        gd[p, -1] = np.float32(np.sum((X[p].astype(np.float64) - X[c]) ** 2))
        o = np.argsort(gd[p], kind="stable")
        gi[p], gd[p] = gi[p][o], gd[p][o]
    elif mistake == "other_leaf":
        c = int(perm[(np.nonzero(perm == p)[0][0] + 700) % len(perm)])
        gi[p, -1] = c
    elif mistake == "distance":
        gd[p, 2] *= np.float32(1.001)
    elif mistake == "duplicate":
        gi[p, 3] = gi[p, 2]
    elif mistake == "order":
        gi[p, [0, 1]] = gi[p, [1, 0]]
        gd[p, [0, 1]] = gd[p, [1, 0]]
    else:
        gi[p, 0] = p
    with pytest.raises(AssertionError):
        check_quant_leaf(X, perm, off, gi, gd, k, kp, oracle.PREC_BF16)


def test_quant_leaf_rejects_a_dropped_near_neighbour(quant_case):
    # the nearest neighbour removed and the rest shifted up, a candidate from
    # the end of the k' list appended: a sure candidate is then missing
    X, perm, off, oi, od, k, kp = quant_case
    gi, gd = oi.copy(), od.copy()
    p = 300
    gi[p, :-1], gd[p, :-1] = oi[p, 1:], od[p, 1:]
    oj, ojd = oracle.leaf_knn_quant(X, perm, off, kp, kp, oracle.PREC_BF16)
    c = int(oj[p, -1])
    gi[p, -1] = c
    gd[p, -1] = np.float32(np.sum((X[p].astype(np.float64) - X[c]) ** 2))
    with pytest.raises(AssertionError):
        check_quant_leaf(X, perm, off, gi, gd, k, kp, oracle.PREC_BF16)


@pytest.fixture(scope="module")
def prop_case():
    X = synthetic.gist_like(1200, 24, centers=5, seed=4)
    k = 8
    lists = np.stack([oracle.leaf_knn(X, *oracle.partition(X, 3, t, 32), k)[0] for t in range(2)])
    mi, md = oracle.merge(X, lists, k)
    pi, pd = oracle.propagate(X, mi, k)
    return X, lists, mi, md, pi, pd, k


def test_rows_accept_the_oracle(prop_case):
    X, lists, mi, md, pi, pd, k = prop_case
    assert check_rows(X, mi, md, mi, md, cands=merge_candidates(lists)) == 0
    assert check_rows(X, pi, pd, pi, pd, cands=propagation_candidates(mi)) == 0


@pytest.mark.parametrize("mistake", ["swap_isolated", "foreign_id", "distance", "profile", "padding"])
def test_rows_reject_planted_mistakes(prop_case, mistake):
    X, lists, mi, md, pi, pd, k = prop_case
    gi, gd = pi.copy(), pd.copy()
    p = 50
    if mistake == "swap_isolated":
        gi[p, [0, 1]] = gi[p, [1, 0]]
    elif mistake == "foreign_id":
        cand = propagation_candidates(mi)(p)
        c = int(np.setdiff1d(np.arange(len(X)), np.append(cand, p))[0])
        gi[p, -1] = c
        gd[p, -1] = np.float32(np.sum((X[p].astype(np.float64) - X[c]) ** 2))
    elif mistake == "distance":
        gd[p, 4] *= np.float32(1 + 1e-4)
    elif mistake == "profile":
        gi[p, -1], gd[p, -1] = mi[p, -1], md[p, -1]
    else:
        gi[p, -1], gd[p, -1] = -1, np.inf
    with pytest.raises(AssertionError):
        check_rows(X, gi, gd, pi, pd, cands=propagation_candidates(mi))
