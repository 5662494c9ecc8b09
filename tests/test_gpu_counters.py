"""Read counters of the propagation rounds: what a first-order round scores
and loads, counted on the device, against the same counts taken on the host
from the round's input lists (no skips apply to a single stage call: every
input entry counts as new)."""
import numpy as np
import pytest

from paper_1307_7852_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_counters_of_a_first_order_round():
    import paper_1307_7852_gb300 as k
    X = synthetic.gist_like(5000, 48, centers=12, seed=7)
    Xd = torch.from_numpy(X).cuda()
    h = k.Handle(0)
    kk = 10
    perm = k.knng_partition(Xd, 2, 64, 3, h=h)
    li, ld = k.knng_leaf_knn(Xd, 2, 64, perm, kk, h=h)
    mi, md = k.knng_merge(li, ld, h=h)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    k.knng_set_propagation_counters(cnt, h)
    k.knng_propagate(Xd, mi, md, 2, h=h)
    torch.cuda.synchronize()
    k.knng_set_propagation_counters(None, h)
    got = cnt.cpu().numpy()
    ids = mi.cpu().numpy()
    rows = slots = 0
    for p in range(ids.shape[0]):
        own = ids[p][ids[p] >= 0]
        nb = own[own != p]
        slots += len(nb) * kk
        c = ids[nb].ravel()
        c = c[(c >= 0) & (c != p)]
        rows += len(np.setdiff1d(np.unique(c), own))
    assert got[0] == rows and got[1] == slots
    # the second round skips pairs scored in the first: it reads less
    assert 0 < got[2] < got[0] and 0 < got[3] < got[1]
