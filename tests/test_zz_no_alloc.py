"""The allocation-free propagation entry point against the regular one.

knng_propagate_noalloc serves callers that cannot allocate device memory on
their call path (a plugin under an application's own memory manager, or a
loop that cannot pay for cudaMalloc's implicit synchronisation).  It must
return exactly what knng_propagate returns; it is called twice in a row,
because every call reuses the library's fixed scratch array and inherits the
previous call's contents.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1307_7852_gb300 import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _graph(X, k, T, g, seed):
    import paper_1307_7852_gb300 as knng
    Xd = torch.from_numpy(X).cuda()
    perm = knng.knng_partition(Xd, T, g, seed)
    li, ld = knng.knng_leaf_knn(Xd, T, g, perm, k)
    mi, md = knng.knng_merge(li, ld)
    return Xd, mi, md


@pytest.mark.parametrize("maker,k,rounds,g", [
    (lambda: synthetic.sift_like(20000, 64, centers=32, seed=41), 10, 3, 64),
    (lambda: synthetic.gist_like(12000, 100, centers=16, seed=42), 16, 2, 64),
    # lists of more than 32 (the two-keys-per-lane kernel; flags of entries
    # 32..63 kept in the array between rounds), n * k near the capacity
    (lambda: synthetic.sift_like(12000, 48, centers=24, seed=43), 40, 3, 128),
    # one round: the input goes straight to the output, no scratch used
    (lambda: synthetic.gist_like(8000, 64, centers=16, seed=44), 12, 1, 64),
    # byte rows
    (lambda: synthetic.sift_like(15000, 32, centers=16, seed=45).astype(np.uint8), 12, 2, 64),
])
def test_noalloc_matches_allocating_entry_point(maker, k, rounds, g):
    import paper_1307_7852_gb300 as knng
    X = maker()
    Xd, mi, md = _graph(X, k, 3, g, 5)
    ri, rd = knng.knng_propagate(Xd, mi, md, rounds)
    torch.cuda.synchronize()
    ref_i, ref_d = ri.cpu().numpy(), rd.cpu().numpy()
    for _ in range(2):
        oi = torch.full_like(mi, -7)
        od = torch.full_like(md, -7.0)
        knng.knng_propagate_noalloc(Xd, mi, md, rounds, ids=oi, dists=od)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(oi.cpu().numpy(), ref_i)
        np.testing.assert_allclose(od.cpu().numpy(), ref_d, rtol=1e-5, atol=0)


def test_noalloc_rejects_requests_above_its_capacity():
    import paper_1307_7852_gb300 as knng
    from paper_1307_7852_gb300 import binding
    n, k = 40000, 20  # n*k above the fixed capacity of 524,288 list entries
    X = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    ids = torch.zeros((n, k), dtype=torch.int32, device="cuda")
    dd = torch.zeros((n, k), dtype=torch.float32, device="cuda")
    rc = binding.lib().knng_propagate_noalloc(ctypes.c_void_p(X.data_ptr()), 0, n, 8, 8, k, 2,
                                              ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dd.data_ptr()),
                                              ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dd.data_ptr()), None)
    assert rc == -7
    with pytest.raises(knng.KnngError):
        knng.binding.knng_propagate_noalloc(X, ids, dd, 2)
