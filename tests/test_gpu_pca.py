"""Random principal-direction splits (Sec. 3.4) on the GPU, through the C
ABI.  Stage isolation: the partition is replayed by the oracle with the
GPU's directions, which must give the identical canonical leaf sets bit for
bit; and every GPU direction is checked against the FP64 Lanczos oracle.  A
few Lanczos steps give a Ritz vector whose direction is ill-determined where
the top Ritz values nearly coincide (FP32 and FP64 then pick different
vectors of the near-degenerate pair), so the check that holds for every node
is on the variance captured: the GPU direction's Rayleigh quotient on the
node's sample covariance must reach the oracle's top Ritz value to within
2e-4 relative (first order in the FP32 rounding of the Lanczos basis times
the Ritz residual), besides unit length and the sign convention."""
import numpy as np
import pytest

import oracle
from oracle import pca
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


CASES = [
    ("sift10k", lambda: synthetic.sift_like(10000, 128, centers=64, seed=1), 3, 64, 7),
    ("gist_d960", lambda: synthetic.gist_like(4000, 960, centers=16, seed=2), 2, 256, 3),
    ("f16_d96", lambda: synthetic.sphere_f16(6000, 96, centers=32, seed=3), 2, 100, 5),
    ("ragged_d7", lambda: synthetic.gaussian_mixture(3000, 7, centers=6, seed=4), 2, 30, 9),
]


@pytest.mark.parametrize("name,mk,T,g,seed", CASES, ids=[c[0] for c in CASES])
def test_pca_partition_replays_and_directions_match(name, mk, T, g, seed):
    X = mk()
    Xf = X.astype(np.float32)
    n, d = X.shape
    perm, dirs = knng().knng_partition_pca(dev(X), T, g, seed, with_dirs=True)
    perm, dirs = host(perm), host(dirs)
    nodes = oracle.split_nodes(n, g)
    cos = []
    for t in range(T):
        # the partition, replayed with the GPU's directions: bit-exact
        p_o, off_o = oracle.partition_with_dirs(Xf, dirs[t], g)
        np.testing.assert_array_equal(perm[t], p_o)
        # every split direction against the FP64 Lanczos oracle
        for (l, v, off, m) in nodes:
            members = np.sort(perm[t][off:off + m])
            a, theta = pca.principal_direction(Xf, members, seed, t, l, v, with_value=True)
            g_dir = dirs[t][2 ** l - 1 + v].astype(np.float64)
            assert abs(np.linalg.norm(g_dir) - 1.0) < 1e-5
            assert g_dir[int(np.argmax(np.abs(g_dir)))] > 0, "sign convention"
            C = pca.sample_covariance(Xf, members, seed, t, l, v)
            rq = float(g_dir @ C @ g_dir) / float(g_dir @ g_dir)
            assert rq >= theta * (1 - 2e-4), (t, l, v, rq, theta)
            cos.append(float(a @ g_dir))
    cos = np.array(cos)
    print(f"directions with cos > 0.999 to the oracle's: {np.mean(cos > 0.999):.4f} of {len(cos)}")
    assert np.median(cos) > 0.99999


def test_pca_build_valid_and_recall_vs_random():
    k = knng()
    X = synthetic.sift_like(20000, 64, centers=64, std=20.0, seed=6)
    Xd = dev(X)
    ids_r, _ = k.knng_build(Xd, 10, 2, 64, 0, 4)
    ids_p, d_p = k.knng_build(Xd, 10, 2, 64, 0, 4, partitioner=k.PART_PCA)
    ids_p, d_p = host(ids_p), host(d_p)
    assert np.all((ids_p >= 0) & (ids_p < 20000))
    assert np.all(np.diff(d_p, axis=1) >= 0)
    q = synthetic.sample_ids(20000, 2000, 1)
    ei, _ = k.knng_exact_knn(Xd, dev(q), 10)
    ei = host(ei)
    rec = lambda ids: np.mean([len(set(ids[p]) & set(ei[r])) / 10 for r, p in enumerate(q)])
    r_rand, r_pca = rec(host(ids_r)), rec(ids_p)
    print(f"recall T=2, no propagation: random {r_rand:.4f}, principal {r_pca:.4f}")
    assert r_pca > r_rand
