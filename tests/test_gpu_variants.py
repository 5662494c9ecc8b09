"""The paper's own propagation and stopping rules on the GPU, through the C
ABI, against the CPU oracle: best-first propagation with a visit budget
(Sec. 3.2), pairwise updating (Sec. 3.4) and divisions added until the
effective rate r_m drops below a threshold (Sec. 3.2, Sec. 4).

Integer-valued (SIFT-like) data makes every distance exact in FP32, so ids
and distances must match exactly; real-valued data follows the FP32
tolerance rule of the other parity tests.
"""
import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic
from test_gpu_parity import assert_valid_rows
from validity import check_rows, propagation_candidates

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
    return Xd, mi, md


# ------------------------------------------------------ best-first (f2) --
@pytest.mark.parametrize("budget", [10, 40, 100, 300])
def test_best_first_integer_exact(budget):
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    Xd, mi, md = _merged(X, 10, 4, 64, 7)
    bi, bd = knng().knng_propagate_best_first(Xd, mi, budget)
    oi, od = oracle.propagate_best_first(X, host(mi), 10, budget)
    np.testing.assert_array_equal(host(bi), oi)
    np.testing.assert_array_equal(host(bd), od)


def test_best_first_two_rounds_and_byte_rows():
    X = synthetic.sift_like(6000, 96, centers=32, seed=2)
    Xd, mi, md = _merged(X, 12, 3, 64, 3)
    oi = host(mi)
    for _ in range(2):
        oi, od = oracle.propagate_best_first(X, oi, 12, 150)
    for Xin in (Xd, dev(X.astype(np.uint8))):
        bi, bd = knng().knng_propagate_best_first(Xin, mi, 150, rounds=2)
        np.testing.assert_array_equal(host(bi), oi)
        np.testing.assert_array_equal(host(bd), od)


@pytest.mark.parametrize("n,d,k,budget", [(5000, 64, 10, 64), (3000, 37, 20, 400)])
def test_best_first_real_valued(n, d, k, budget):
    X = synthetic.gist_like(n, d, centers=16, seed=n)
    Xd, mi, md = _merged(X, k, 3, max(96, 2 * k + 2), 4)
    bi, bd = knng().knng_propagate_best_first(Xd, mi, budget)
    oi, od = oracle.propagate_best_first(X, host(mi), k, budget)
    # the queue order is decided by the canonical FP32 distance on both
    # sides, so the visited sets agree; the lists follow the FP32 rule
    check_rows(X, host(bi), host(bd), oi, od)
    assert_valid_rows(host(bi), host(bd), n)


# ---------------------------------------------------- pairwise (f3) -----
def test_pairwise_integer_exact_one_and_three_rounds():
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    Xd, mi, md = _merged(X, 10, 4, 64, 7)
    pi, pd = knng().knng_propagate_pairwise(Xd, mi, md, 1)
    oi, od = oracle.propagate_pairwise(X, host(mi), 10)
    np.testing.assert_array_equal(host(pi), oi)
    np.testing.assert_array_equal(host(pd), od)
    # rounds 2 and 3 skip the pairs scored before; the result must equal
    # three plain oracle rounds
    qi, qd = knng().knng_propagate_pairwise(Xd, mi, md, 3)
    oi = host(mi)
    for _ in range(3):
        oi, od = oracle.propagate_pairwise(X, oi, 10)
    np.testing.assert_array_equal(host(qi), oi)
    np.testing.assert_array_equal(host(qd), od)
    knng().knng_sync()


def test_pairwise_real_valued_and_better_than_first_order():
    X = synthetic.gist_like(6000, 96, centers=16, seed=6)
    Xd, mi, md = _merged(X, 16, 3, 96, 4)
    pi, pd = knng().knng_propagate_pairwise(Xd, mi, md, 1)
    oi, od = oracle.propagate_pairwise(X, host(mi), 16)
    # candidates of p: C(p) and every q with p in C(q)
    m_h = host(mi)
    fwd = propagation_candidates(m_h)
    cand = [set(fwd(p).tolist()) - {p} for p in range(m_h.shape[0])]
    rev = [set() for _ in cand]
    for q, cq in enumerate(cand):
        for p in cq:
            rev[p].add(q)
    check_rows(X, host(pi), host(pd), oi, od, cands=lambda p: np.array(sorted(cand[p] | rev[p])))
    fi, fd = knng().knng_propagate(Xd, mi, md, 1)
    assert np.all(host(pd) <= host(fd) * (1 + 1e-6))


# ------------------------------------------------- r_m trigger (Sec. 4) --
@pytest.mark.parametrize("r_stop", [0.05, 0.2])
def test_adaptive_divisions_match_oracle(r_stop):
    X = synthetic.sift_like(10000, 128, centers=64, seed=1)
    gi, gd = knng().knng_build(dev(X), 10, 16, 64, 1, 7, r_stop=r_stop)
    m, rates = knng().knng_divisions_used()
    info = {}
    oi, od = oracle.build_graph(X, 10, 16, 64, 1, 7, r_stop=r_stop, info=info)
    assert m == info["divisions"]
    np.testing.assert_allclose(rates, info["rates"], rtol=1e-6, atol=1e-7)
    np.testing.assert_array_equal(host(gi), oi)
    np.testing.assert_array_equal(host(gd), od)
    # the adaptive graph is the plain build with the divisions it used
    pi, pd = knng().knng_build(dev(X), 10, m, 64, 1, 7)
    np.testing.assert_array_equal(host(pi), oi)


def test_paper_configuration_end_to_end():
    # Sec. 4's settings: divisions until r_m < 0.05, then best-first
    # propagation (budget 100); and the same with pairwise updating rounds
    X = synthetic.sift_like(8000, 64, centers=48, seed=9)
    k = knng()
    gi, gd = k.knng_build(dev(X), 10, 12, 64, 2, 5, r_stop=0.05, propagation=k.PROP_BEST_FIRST, budget=100)
    oi, od = oracle.build_graph(X, 10, 12, 64, 2, 5, r_stop=0.05, prop=oracle.PROP_BEST_FIRST, budget=100)
    np.testing.assert_array_equal(host(gi), oi)
    np.testing.assert_array_equal(host(gd), od)
    gi, gd = k.knng_build(dev(X), 10, 4, 64, 2, 5, propagation=k.PROP_PAIRWISE)
    oi, od = oracle.build_graph(X, 10, 4, 64, 2, 5, prop=oracle.PROP_PAIRWISE)
    np.testing.assert_array_equal(host(gi), oi)
    np.testing.assert_array_equal(host(gd), od)


def test_batched_variants():
    k = knng()
    Xs = [synthetic.sift_like(n, 32, centers=8, seed=n) for n in (3000, 4500)]
    for prop, budget in ((k.PROP_BEST_FIRST, 60), (k.PROP_PAIRWISE, 0)):
        outs = k.knng_build_batched([dev(X) for X in Xs], 8, 3, 48, 2, 4, propagation=prop, budget=budget)
        for X, (bi, bd) in zip(Xs, outs):
            si, sd = k.knng_build(dev(X), 8, 3, 48, 2, 4, propagation=prop, budget=budget)
            np.testing.assert_array_equal(host(bi), host(si))
            np.testing.assert_array_equal(host(bd), host(sd))
    with pytest.raises(k.KnngError):
        k.knng_build_batched([dev(X) for X in Xs], 8, 3, 48, 1, 4, r_stop=0.05)
