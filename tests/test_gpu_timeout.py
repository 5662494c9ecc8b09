"""Bounded device waits: a wait that runs out is reported, not hung on.

The tensor-core leaf kernel waits (bounded) for its TMA copies and for its
MMAs to release pipeline stages.  With a limit of a few cycles those waits
give up on copies that are still in flight: every CTA then records the
failure, drains its own copies and MMAs under the one-second limit, frees its
tensor memory and returns; knng_sync reports KNNG_ERR_TIMEOUT, and the same
handle computes the right graph once the default limit is back."""
import numpy as np
import pytest

import oracle
from paper_1307_7852_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KNNG_ERR_TIMEOUT = -5


def test_wait_limit_runs_out_and_the_context_survives():
    import paper_1307_7852_gb300 as k
    X = synthetic.sift_like(12000, 128, centers=32, seed=4)
    Xd = torch.from_numpy(X).cuda()
    h = k.Handle(0)
    T, g, kk, seed = 2, 128, 10, 3
    perm = k.knng_partition(Xd, T, g, seed, h=h)
    k.knng_sync(h)
    k.knng_set_wait_limit(8, h)
    k.knng_leaf_knn(Xd, T, g, perm, kk, k.PREC_BF16, 2, h=h)
    with pytest.raises(k.KnngError) as e:
        k.knng_sync(h)
    assert e.value.code == KNNG_ERR_TIMEOUT
    # the flag was cleared; the default limit computes the right lists
    k.knng_set_wait_limit(0, h)
    ids, dd = k.knng_leaf_knn(Xd, T, g, perm, kk, k.PREC_BF16, 2, h=h)
    k.knng_sync(h)
    perm_h, ids, dd = perm.cpu().numpy(), ids.cpu().numpy(), dd.cpu().numpy()
    off = k.knng_leaf_offsets(12000, g)
    for t in range(T):
        oi, od = oracle.leaf_knn(X, perm_h[t], off, kk)
        np.testing.assert_array_equal(ids[t], oi)
        np.testing.assert_array_equal(dd[t], od)
    with pytest.raises(k.KnngError):
        k.knng_set_wait_limit(-1, h)
