"""Complete per-row validity checks of GPU k-NN lists against the oracle.

Where several lists are correct -- distances that tie within the FP32
tolerance, or a reduced-precision candidate stage whose FP32-accumulated
distances order near-equal candidates differently from FP64 -- a GPU row may
differ from the oracle's.  These helpers check EVERY row: a row that differs
passes only if the difference is one the arithmetic allows.

FP32 stages (a top-k of a known candidate set by exact distance):
  * ids distinct, not the point itself, drawn from the candidate set, padding
    (-1, +inf) only after the real entries;
  * every listed distance within 1e-5 relative of the FP64 distance of that
    pair (the entry is real);
  * the sorted distance profile within 1e-5 relative of the oracle's, position
    by position, and ids equal wherever the oracle's neighbouring distances
    differ by more than 1e-5 relative (the tie rule of the FP32 parity bar).

Reduced-precision leaf stage (top-k' by the quantised distance D~, then the
exact top-k of those): with e_pj a bound on the GPU's error in D~(p, j),
every candidate j with D~_pj < tau - 2e (tau the k'-th smallest D~ of the
row, e the row's largest bound) is surely among the GPU's k' candidates and
every j with D~_pj > tau + 2e surely not; the GPU row must then
  * hold only sure or band candidates, with real distances (1e-5 rule);
  * contain every sure candidate whose exact distance is below its k-th
    distance (by more than 1e-5 relative);
  * be completable to k' candidates: the sure ones, its own, and band
    candidates no nearer than its k-th distance.
"""
from __future__ import annotations

import numpy as np

import oracle

REL = 1e-5


def _row_dists(Xr, p, ids, cosine=False):
    diff = Xr[ids].astype(np.float64) - Xr[p].astype(np.float64)
    d = np.einsum("ij,ij->i", diff, diff)
    return d * 0.5 if cosine else d


def rows_of(X, cosine=False):
    """The rows the distances are taken on (unit rows for the cosine metric)."""
    X = np.asarray(X)
    if X.dtype == np.float16:
        X = X.astype(np.float32)
    return oracle.normalize_rows(X) if cosine else np.ascontiguousarray(X, dtype=np.float32)


def check_rows(X, gi, gd, oi, od, rows=None, cands=None, cosine=False, rel=REL):
    """Complete check of GPU rows (gi, gd) against oracle rows (oi, od) of an
    FP32 top-k stage.  rows: the point of each row (default 0..n-1); cands:
    callable(row index) -> allowed ids, or None."""
    Xr = rows_of(X, cosine)
    gi = np.asarray(gi).reshape(-1, np.asarray(gi).shape[-1])
    gd = np.asarray(gd).reshape(gi.shape).astype(np.float64)
    oi = np.asarray(oi).reshape(gi.shape)
    od = np.asarray(od).reshape(gi.shape).astype(np.float64)
    n_rows, k = gi.shape
    rows = np.arange(n_rows) if rows is None else np.asarray(rows)
    fin = np.isfinite(od)
    assert np.array_equal(np.isfinite(gd), fin), "padding differs"
    assert np.array_equal(gi < 0, ~fin), "padding ids"
    # positional distance profile
    tol = rel * np.maximum(np.abs(od[fin]), 1e-30)
    err = np.abs(gd[fin] - od[fin])
    assert np.all(err <= tol), f"distance profile off by {np.max(err / np.maximum(od[fin], 1e-30)):.3g} relative"
    # ids at isolated positions
    left = np.full(od.shape, np.inf)
    left[:, 1:] = (od[:, 1:] - od[:, :-1]) / np.maximum(od[:, 1:], 1e-30)
    right = np.full(od.shape, np.inf)
    right[:, :-1] = (od[:, 1:] - od[:, :-1]) / np.maximum(od[:, 1:], 1e-30)
    right[:, k - 1] = 0.0  # the next oracle candidate is not visible: the last slot may tie
    iso = (left > rel) & (right > rel)
    mism = iso & (gi != oi)
    assert not mism.any(), f"{mism.sum()} isolated positions differ"
    # every entry of a row that differs anywhere is real, distinct, allowed
    diff_rows = np.nonzero(np.any(gi != oi, axis=1))[0]
    for r in diff_rows:
        p = int(rows[r])
        v = gi[r][gi[r] >= 0]
        assert len(np.unique(v)) == len(v), f"row {r}: repeated ids"
        assert not np.any(v == p), f"row {r}: the point itself"
        if cands is not None:
            allowed = np.asarray(cands(r))
            assert np.all(np.isin(v, allowed)), f"row {r}: id outside the candidate set"
        true = _row_dists(Xr, p, v, cosine)
        g = gd[r][: len(v)]
        assert np.all(np.abs(g - true) <= rel * np.maximum(true, 1e-30)), f"row {r}: listed distance not the pair's"
    return len(diff_rows)


def gram_error_bound(nq_p, nq_j, absdot, d, extra_roundings=4):
    """Bound on |D~_GPU - D~| for D~ = |x|^2 + |y|^2 - 2 x.y of quantised rows
    whose products are exact in FP32 (BF16 x BF16, E4M3 x E4M3): each of the
    d FP32 additions of the dot product and of each norm errs by at most one
    unit of 2^-22 relative (a unit of slack over round-to-nearest for the
    tensor core's accumulation order), plus the final combination."""
    u = 2.0 ** -22
    return (d + extra_roundings) * u * (nq_p + nq_j + 2.0 * absdot)


def check_quant_leaf(X, perm, off, gi, gd, k, kp, prec, rel=REL):
    """Complete check of one tree's reduced-precision leaf graph (the GPU's
    knng_leaf_knn output rows gi/gd [n, k]) on the leaf layout (perm, off).
    prec: oracle.PREC_BF16 / PREC_FP8E4M3 (quantised candidate stage) or
    PREC_FP32 (FP32 Gram candidate stage, rows unquantised)."""
    Xf = rows_of(X)
    n, d = Xf.shape
    if prec == oracle.PREC_FP32:
        Xq = Xf.astype(np.float64)
        sc = np.ones(n)
        Q = Xq
    else:
        Xq, sc = oracle.quantize_rows(Xf, prec)
        sc = sc.astype(np.float64)
        Q = Xq / sc[:, None]          # the codes (E4M3) or the bfloat16 values
    gi = np.asarray(gi)
    gd = np.asarray(gd).astype(np.float64)
    checked_band = 0
    for L in range(len(off) - 1):
        mem = np.asarray(perm[off[L]:off[L + 1]])
        m = len(mem)
        A = Xq[mem]
        nq = np.einsum("ij,ij->i", Q[mem], Q[mem])
        Dq = (np.einsum("ij,ij->i", A, A)[:, None] + np.einsum("ij,ij->i", A, A)[None, :] - 2.0 * A @ A.T)
        absdot = np.abs(Q[mem]) @ np.abs(Q[mem]).T
        s2 = sc[mem] ** 2
        bound = gram_error_bound((s2 * nq)[:, None], (s2 * nq)[None, :],
                                 np.outer(sc[mem], sc[mem]) * absdot, d)
        for a in range(m):
            p = int(mem[a])
            row_i, row_d = gi[p], gd[p]
            others = np.array([b for b in range(m) if b != a])
            want = min(k, m - 1)
            v = row_i[row_i >= 0]
            assert len(v) == want, f"point {p}: {len(v)} entries, {want} expected"
            assert np.all(row_i[want:] == -1) and np.all(np.isinf(row_d[want:]))
            assert len(np.unique(v)) == len(v) and not np.any(v == p), f"point {p}: bad ids"
            assert np.all(np.isin(v, mem)), f"point {p}: id outside its leaf"
            true = _row_dists(Xf, p, v)
            g = row_d[:want]
            assert np.all(np.abs(g - true) <= rel * np.maximum(true, 1e-30)), f"point {p}: distance not the pair's"
            assert np.all(np.diff(g) >= 0), f"point {p}: not sorted"
            kth = g[-1]
            if m - 1 <= kp:
                # every member is a candidate: the exact top-k of the leaf
                sure = others
                band = np.array([], dtype=np.int64)
            else:
                dq = Dq[a, others]
                order = np.lexsort((mem[others], dq))
                tau = dq[order[kp - 1]]
                e = np.max(bound[a, others])
                sure = others[dq < tau - 2 * e]
                band = others[np.abs(dq - tau) <= 2 * e]
                assert len(sure) <= kp
                checked_band += len(band) > 0
            loc = {int(mem[b]): b for b in range(m)}
            vb = np.array([loc[int(x)] for x in v])
            in_sure_or_band = np.isin(vb, np.concatenate([sure, band]))
            assert np.all(in_sure_or_band), f"point {p}: an id that cannot be among the {kp} candidates"
            # sure candidates nearer than the row's k-th must be listed
            ds = _row_dists(Xf, p, mem[sure]) if len(sure) else np.zeros(0)
            missing = (ds < kth * (1 - rel)) & ~np.isin(sure, vb)
            assert not missing.any(), f"point {p}: a sure candidate nearer than its k-th is missing"
            if m - 1 > kp:
                # completable to kp candidates without a band candidate that
                # would have beaten the row's k-th
                extra = np.setdiff1d(band, np.concatenate([sure, vb]))
                de = _row_dists(Xf, p, mem[extra]) if len(extra) else np.zeros(0)
                fill = int(np.sum(de >= kth * (1 - rel)))
                used = len(np.union1d(sure, vb))
                assert used <= kp and used + fill >= kp, f"point {p}: no consistent candidate set"
    return checked_band


def merge_candidates(leaf_ids):
    """cands(p) for the merge stage: the union of p's T leaf lists."""
    L = np.asarray(leaf_ids)

    def cands(p):
        v = L[:, p, :].ravel()
        return np.unique(v[v >= 0])
    return cands


def propagation_candidates(ids_in, rows=None):
    """cands(r) for a first-order round: N(p) and its neighbours' lists."""
    ids_in = np.asarray(ids_in)
    rows = np.arange(ids_in.shape[0]) if rows is None else np.asarray(rows)

    def cands(r):
        p = int(rows[r])
        own = ids_in[p][ids_in[p] >= 0]
        v = np.concatenate([own, ids_in[own].ravel()])
        return np.unique(v[v >= 0])
    return cands


def check_build_stagewise(knng, torch, X, k, T, g, R, seed, gi, gd, precision=0, cosine=False, net=None,
                          learned="features"):
    """A whole GPU build (gi, gd) checked through its stages: the build must
    equal the composition of the GPU's stage entry points bit for bit, and
    every stage, fed the GPU's previous-stage output, must pass the complete
    check against the oracle stage fed the same input.  net: a learned
    network; learned = "features" (per-level feature splits,
    knng_partition_learned) or "embedding" (random trees on the network's
    outputs z)."""
    Xh = np.asarray(X)
    Xd = torch.from_numpy(np.ascontiguousarray(Xh)).cuda()
    Xr = rows_of(Xh, cosine)
    Ud = knng.knng_normalize_rows(Xd) if cosine else Xd
    if cosine:
        np.testing.assert_array_equal(Ud.cpu().numpy(), Xr)
    if net is not None and learned == "features":
        perm, Z = knng.knng_partition_learned(net, Xd, T, g, seed, with_z=True)
        Zh = Z.cpu().numpy()
    elif net is not None:
        Z = knng.knng_mlp_forward(net, Xd)
        perm = knng.knng_partition(Z, T, g, seed)
        Zh = Z.cpu().numpy()
    else:
        perm = knng.knng_partition(Ud, T, g, seed)
    li, ld = knng.knng_leaf_knn(Ud, T, g, perm, k, precision, 2)
    cur_i, cur_d = knng.knng_merge(li, ld)
    stages = [(cur_i, cur_d)]
    for _ in range(R):
        cur_i, cur_d = knng.knng_propagate(Ud, cur_i, cur_d, 1)
        stages.append((cur_i, cur_d))
    torch.cuda.synchronize()
    half = np.float32(0.5) if cosine else np.float32(1.0)
    np.testing.assert_array_equal(np.asarray(gi), cur_i.cpu().numpy())
    np.testing.assert_array_equal(np.asarray(gd), cur_d.cpu().numpy() * half)
    perm_h = perm.cpu().numpy()
    li_h, ld_h = li.cpu().numpy(), ld.cpu().numpy()
    off = knng.knng_leaf_offsets(Xh.shape[0], g)
    for t in range(T):
        if net is not None and learned == "features":
            op, oo = oracle.partition_features(Xh, Zh, seed, t, g)
        elif net is not None:
            op, oo = oracle.partition(Zh, seed, t, g)
        else:
            op, oo = oracle.partition(Xr, seed, t, g)
        np.testing.assert_array_equal(perm_h[t], op)
        if precision == 0 and not np.all(Xr == np.rint(Xr)):
            check_quant_leaf(Xr, perm_h[t], off, li_h[t], ld_h[t], k, 2 * k, oracle.PREC_FP32)
        elif precision == 0:
            oi, od = oracle.leaf_knn(Xr, perm_h[t], off, k)
            np.testing.assert_array_equal(li_h[t], oi)
            np.testing.assert_array_equal(ld_h[t], od)
        else:
            check_quant_leaf(Xr, perm_h[t], off, li_h[t], ld_h[t], k, 2 * k, precision)
    prev = li_h
    oi, od = oracle.merge(Xr, li_h, k)
    mi, md = stages[0][0].cpu().numpy(), stages[0][1].cpu().numpy()
    check_rows(Xr, mi, md, oi, od, cands=merge_candidates(li_h))
    prev = mi
    for r in range(R):
        pi, pd = stages[r + 1][0].cpu().numpy(), stages[r + 1][1].cpu().numpy()
        oi, od = oracle.propagate(Xr, prev, k)
        check_rows(Xr, pi, pd, oi, od, cands=propagation_candidates(prev))
        prev = pi
