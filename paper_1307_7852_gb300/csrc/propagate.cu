// Neighbourhood propagation (Sec. 3.2 of arXiv:1307.7852), in the first-order
// form analysed by Theorem 1: in one synchronous round every point p takes
// the k best of its own list and of the lists of its neighbours, without p.
//
// One warp per point.
//  * Candidates: the k*k ids of the neighbours' lists are fetched with the
//    lanes spread over (neighbour, slot) pairs, and deduplicated in a
//    shared-memory hash set (the per-point replacement of the paper's hash
//    table of evaluated pairs, Sec. 3.4 "Speedup").  Ids already in p's list
//    keep their distance.
//  * Skipping pairs scored before (exact): with per-entry "new" flags from
//    the previous round, a candidate c of a neighbour q is skipped when q was
//    already in p's previous list and c already in q's previous list.  Then c
//    was a candidate of p in the previous round, so either c is in p's list
//    or k listed points beat it, and it cannot enter the new list.
//  * Skipping pairs that shared a leaf (exact, first round after the merge):
//    when every leaf list was the exact k best of its leaf, the merge marks
//    each entry with the trees whose lists held it.  If p's entry q and q's
//    entry c share a tree t, then p, q and c were in one leaf of tree t, so c
//    is in p's tree-t list or k points of that leaf beat it; either way c is
//    in p's merged list or cannot enter the new one, and is skipped.
//  * Scoring: 16 candidates at a time by warp_canon_dist16 (coalesced 16-byte
//    row loads, 16 rows in flight per warp, bit-identical canonical FP32);
//    float rows holding only bytes are scored on their exact byte copy in
//    integer arithmetic (4-byte loads, the same values).
//  * The k best by (dist, id): warp radix select and a warp bitonic sort; the
//    output flags mark the entries that were not in p's input list.
#include "knng_common.cuh"
#include "knng_internal.h"

// Blocks of 256 threads the register budget is sized for (2: 128 registers,
// no spills; 3: 80 registers with small spills, 24 resident warps).
#ifndef KNNG_PROP_MINBLOCKS
#define KNNG_PROP_MINBLOCKS 2
#endif

namespace knng {

struct PropLayout {
    int H;       // hash slots (power of two)
    int hshift;  // 32 - log2(H)
    int cap;     // candidate capacity = k + k*k
    size_t per_warp;
};

static PropLayout prop_layout(int k)
{
    PropLayout L;
    L.cap = k + k * k;
    int H = 64;
    while (H < 2 * (L.cap + 1)) H <<= 1;
    L.H = H;
    int lg = 0;
    while ((1 << lg) < H) ++lg;
    L.hshift = 32 - lg;
    // tab[H] | cid[cap] | cd[cap] | hist[256] | sel[64] | own[64] | own_fl[64] (u64) | keys[192] (u64) |
    // own_tm[64]
    L.cap = (L.cap + 1) & ~1;  // keeps own_fl 8-byte aligned
    L.per_warp = sizeof(int) * (size_t)H + (sizeof(int) + sizeof(float)) * (size_t)L.cap +
                 sizeof(uint32_t) * 256 + sizeof(int) * 64 + sizeof(int) * 64 + sizeof(unsigned long long) * 64 +
                 sizeof(unsigned long long) * 192 + sizeof(int) * 64;
    L.per_warp = (L.per_warp + 15) & ~(size_t)15;
    return L;
}

// kMode: 1 = the first round after the merge, with the merge's tree masks
// and no flags; 2 = a later first-order round, with flags; 0 = any other
// (flags optional, pairwise offers possible).  Separate instantiations, so
// no round carries the code of the others.
template <int E, int kDT, int kMode>
__global__ void __launch_bounds__(256, KNNG_PROP_MINBLOCKS) propagate_kernel(RowLoader<kDT> L, RowLoader<kDtU8> Lb,
                                 const int* __restrict__ xb_bad, const uint8_t* __restrict__ lane_X,
                                 int64_t lane_ld, PairOffers po, int64_t n, int k,
                                 const int32_t* __restrict__ order,
                                 const int32_t* __restrict__ ids_in, const float* __restrict__ d_in,
                                 const unsigned long long* __restrict__ flags_in,
                                 const uint8_t* __restrict__ tm_in, int32_t* __restrict__ ids_out,
                                 float* __restrict__ d_out, unsigned long long* __restrict__ flags_out, int H,
                                 int hshift, int cap, int per_warp_bytes, unsigned long long* __restrict__ stats)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char* base = smem_raw + (size_t)w * per_warp_bytes;
    int* tab = reinterpret_cast<int*>(base);
    int* cid = tab + H;
    float* cd = reinterpret_cast<float*>(cid + cap);
    uint32_t* hist = reinterpret_cast<uint32_t*>(cd + cap);
    int* sel = reinterpret_cast<int*>(hist + 256);
    int* own = sel + 64;
    unsigned long long* own_fl = reinterpret_cast<unsigned long long*>(own + 64);
    uint64_t* keys = reinterpret_cast<uint64_t*>(own_fl + 64);
    int* own_tm = reinterpret_cast<int*>(keys + 192);
    const uint32_t hmask = (uint32_t)H - 1;
    const int kk = k * k;
    // float rows with an exact byte copy: score on the copy (same values)
    bool bytes = false;
    if constexpr (kDT == kDtF32) bytes = xb_bad && *xb_bad == 0;

    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long n_rows = 0, n_slots = 0;  // what this lane read (stats)
    const bool use_flags = kMode == 2 || (kMode == 0 && flags_in != nullptr);
    // The warp's next point, its own list, flags and tree masks are fetched
    // while the current point is processed (and the point after it is
    // looked up in the order), so a point starts with them in registers.
    auto point_at = [&](int64_t w2) -> int32_t {
        return w2 < n ? (order ? order[w2] : (int32_t)w2) : -1;
    };
    int32_t nid[E], ntm[E];
    float nd[E];
    unsigned long long npf = ~0ull;
    // and, with flags, once its list has arrived (fetched half way through
    // a point), the flags of its neighbours' lists
    unsigned long long nfl[E];
    bool have_next = false;  // nfl holds the current point's
    auto fetch_neigh = [&]() {
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int e = 32 * q + lane;
            const int32_t id = (e < k && nid[q] < n) ? nid[q] : -1;
            nfl[q] = id >= 0 ? flags_in[id] : 0ull;
        }
    };
    auto fetch = [&](int32_t p2) {
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int e = 32 * q + lane;
            const bool v = p2 >= 0 && e < k;
            nid[q] = v ? ids_in[(int64_t)p2 * k + e] : -1;
            nd[q] = v ? d_in[(int64_t)p2 * k + e] : 0.f;
            ntm[q] = (kMode == 1 && v) ? (int)tm_in[(int64_t)p2 * k + e] : 0;
        }
        npf = (use_flags && p2 >= 0) ? flags_in[p2] : ~0ull;
    };
    int32_t p_next = point_at(gw), p_next2 = point_at(gw + nw);
    fetch(p_next);
    for (int64_t wi = gw; wi < n; wi += nw) {
        const int32_t p = p_next;
        int32_t myid[E], mytm[E];
        float myd[E];
#pragma unroll
        for (int q = 0; q < E; ++q) {
            myid[q] = nid[q];
            myd[q] = nd[q];
            mytm[q] = ntm[q];
        }
        const unsigned long long pf = npf;
        unsigned long long myfl[E];
        const bool have = have_next;
#pragma unroll
        for (int q = 0; q < E; ++q) myfl[q] = nfl[q];
        have_next = false;
        p_next = p_next2;
        p_next2 = point_at(wi + 2 * nw);
        fetch(p_next);
        for (int s = lane * 4; s < H; s += 128) *reinterpret_cast<int4*>(tab + s) = make_int4(-1, -1, -1, -1);
        __syncwarp();
        if (lane == 0) hash_insert(tab, (uint32_t)hshift, hmask, p);
        __syncwarp();
        // p's own list: ids keep their distances
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int e = 32 * q + lane;
            int32_t id = -1;
            float dd = 0.f;
            if (e < k) {
                id = myid[q];
                dd = myd[q];
                if (id >= n) id = -1;  // ids outside [0, n) are treated as empty slots
                own[e] = id;
                if (kMode == 1) own_tm[e] = mytm[q];
            }
            const bool ins = id >= 0 && hash_insert(tab, (uint32_t)hshift, hmask, id);
            const uint32_t b = __ballot_sync(KNNG_FULL_MASK, ins);
            if (ins) {
                const int pos = cnt + __popc(b & lanemask_lt());
                cid[pos] = id;
                cd[pos] = dd;
            }
            cnt += __popc(b);
        }
        const int nknown = cnt;
        // flags of the neighbours' lists (entries of a list that are new)
        if (use_flags) {
            if (have) {
#pragma unroll
                for (int q = 0; q < E; ++q)
                    if (32 * q + lane < k) own_fl[32 * q + lane] = myfl[q];
            } else {
                for (int e = lane; e < k; e += 32) {
                    const int32_t q = own[e];
                    own_fl[e] = q >= 0 ? flags_in[q] : 0ull;
                }
            }
        }
        __syncwarp();
        constexpr int G = 4;  // list loads in flight per lane before the hash inserts
        // The live slots are listed first, (e << 8) | f, so the loop below
        // runs over them only: with flags, q new in p's list or c new in q's
        // (a later round loads about a third of the k*k slots); in the first
        // round, c not sharing an exact leaf with p and q (the lane of
        // neighbour q reads q's k tree masks, and only the live ids are
        // loaded)
        int nlive = -1;  // no list: the loop over all slots below
        // the list sits in the candidate-distance array past p's own entries
        // (free until the scoring, room for all k*k slots)
        int* live = reinterpret_cast<int*>(cd) + nknown;
        if (use_flags || kMode == 1) {
            const unsigned long long kmask = k >= 64 ? ~0ull : ((1ull << k) - 1ull);
            nlive = 0;
            for (int e0 = 0; e0 < k; e0 += 32) {
                const int e = e0 + lane;
                unsigned long long msk = 0ull;
                if (e < k) {
                    const int32_t q = own[e];
                    if (q >= 0 && q != p) {
                        const int ot = kMode == 1 ? own_tm[e] : 0;
                        if (ot == 0) {
                            // no shared leaf known (or no masks: some leaf
                            // was not exact): every slot, and with flags the
                            // new ones
                            msk = (!use_flags || ((pf >> e) & 1ull)) ? kmask : (own_fl[e] & kmask);
                        } else {
                            const uint8_t* tq = tm_in + (int64_t)q * k;
                            if ((k & 3) == 0) {
                                for (int f0 = 0; f0 < k; f0 += 4) {
                                    const uint32_t w4 = *reinterpret_cast<const uint32_t*>(tq + f0);
#pragma unroll
                                    for (int b = 0; b < 4; ++b)
                                        if ((((w4 >> (8 * b)) & 0xFFu) & (uint32_t)ot) == 0u) msk |= 1ull << (f0 + b);
                                }
                            } else {
                                for (int f = 0; f < k; ++f)
                                    if ((tq[f] & ot) == 0) msk |= 1ull << f;
                            }
                        }
                    }
                }
                const int c = __popcll(msk);
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(KNNG_FULL_MASK, incl, o);
                    if (lane >= o) incl += t;
                }
                int j = nlive + incl - c;
                nlive += __shfl_sync(KNNG_FULL_MASK, incl, 31);
                while (msk) {
                    live[j++] = (e << 8) | (__ffsll((long long)msk) - 1);
                    msk &= msk - 1ull;
                }
            }
            __syncwarp();
        }
        if (nlive >= 0) {
            for (int i0 = 0; i0 < nlive; i0 += 32 * G) {
                int32_t o[G];
#pragma unroll
                for (int gi = 0; gi < G; ++gi) {
                    o[gi] = -1;
                    const int i = i0 + 32 * gi + lane;
                    if (i < nlive) {
                        const int v = live[i];
                        o[gi] = ids_in[(int64_t)own[v >> 8] * k + (v & 255)];
                        if (stats) ++n_slots;
                    }
                }
#pragma unroll
                for (int gi = 0; gi < G; ++gi) {
                    const int32_t oo = o[gi] < n ? o[gi] : -1;
                    const bool ins = oo >= 0 && hash_insert(tab, (uint32_t)hshift, hmask, oo);
                    const uint32_t b = __ballot_sync(KNNG_FULL_MASK, ins);
                    if (ins) cid[cnt + __popc(b & lanemask_lt())] = oo;
                    cnt += __popc(b);
                }
            }
        }
        // otherwise lanes over (neighbour e, slot f) with
        // i = e*k + f = lane + 32*step, advanced without division
        int e = lane / k, f = lane - (lane / k) * k;
        const int de = 32 / k, df = 32 - (32 / k) * k;
        for (int i0 = 0; i0 < (nlive >= 0 ? 0 : kk); i0 += 32 * G) {
            int32_t o[G];
#pragma unroll
            for (int gi = 0; gi < G; ++gi) {
                o[gi] = -1;
                if (i0 + 32 * gi + lane < kk) {
                    const int32_t q = own[e];
                    if (q >= 0 && q != p) {
                        const bool qnew = (pf >> e) & 1ull;
                        const bool cnew = use_flags ? ((own_fl[e] >> f) & 1ull) : true;
                        if (qnew || cnew) {
                            // c of q is useless when p, q and c shared an
                            // exact leaf: c then is in p's merged list or
                            // k listed points beat it
                            int32_t c = ids_in[(int64_t)q * k + f];
                            if (stats) ++n_slots;
                            if (kMode == 1 && (own_tm[e] & (int)tm_in[(int64_t)q * k + f])) c = -1;
                            o[gi] = c;
                        }
                    }
                }
                e += de;
                f += df;
                if (f >= k) { f -= k; ++e; }
            }
#pragma unroll
            for (int gi = 0; gi < G; ++gi) {
                const int32_t oo = o[gi] < n ? o[gi] : -1;
                const bool ins = oo >= 0 && hash_insert(tab, (uint32_t)hshift, hmask, oo);
                const uint32_t b = __ballot_sync(KNNG_FULL_MASK, ins);
                if (ins) cid[cnt + __popc(b & lanemask_lt())] = oo;
                cnt += __popc(b);
            }
        }
        __syncwarp();
        // the next point's list has arrived by now: fetch its neighbours'
        // flags
        if (use_flags && p_next >= 0) {
            fetch_neigh();
            have_next = true;
        }
        if (stats && lane == 0) n_rows += (unsigned long long)(cnt - nknown);
        // score the new candidates, 32 at a time
        if (lane_X && (kDT == kDtU8 || bytes)) {
            // byte rows, d <= 128: eight lanes per candidate
            const uint4 q = load_query_u8(lane_X, lane_ld, p, L.d);
            for (int c0 = nknown; c0 < cnt; c0 += 32)
                score_u8_g8(lane_X, lane_ld, L.d, q, cid + c0, min(32, cnt - c0), cd + c0);
        } else {
            for (int c0 = nknown; c0 < cnt; c0 += 32) {
                const int nb = min(32, cnt - c0);
                float dd;
                if (kDT == kDtF32 && bytes) dd = warp_canon_dist32(Lb, p, cid + c0, nb);
                else dd = warp_canon_dist32(L, p, cid + c0, nb);
                if (lane < nb) cd[c0 + lane] = dd;
            }
        }
        __syncwarp();
        if (kMode == 0 && po.tgt) {
            // pairwise updating: offer p to every candidate c whose input
            // list it would enter, i.e. (D, p) below c's k-th (dist, id)
            for (int i0 = 0; i0 < cnt; i0 += 32) {
                const int i = i0 + lane;
                bool emit = false;
                int32_t c = -1;
                uint64_t kk = 0;
                if (i < cnt) {
                    c = cid[i];
                    kk = pack_key(cd[i], (uint32_t)p);
                    const int32_t last = ids_in[(int64_t)c * k + k - 1];
                    const uint64_t thr =
                        (last < 0 || last >= n) ? kKeyMax : pack_key(d_in[(int64_t)c * k + k - 1], (uint32_t)last);
                    emit = kk < thr;
                }
                const uint32_t b = __ballot_sync(KNNG_FULL_MASK, emit);
                if (b) {
                    unsigned long long slot0 = 0;
                    if (lane == 0) slot0 = atomicAdd(po.count, (unsigned long long)__popc(b));
                    slot0 = __shfl_sync(KNNG_FULL_MASK, slot0, 0);
                    if (emit) {
                        const unsigned long long slot = slot0 + __popc(b & lanemask_lt());
                        if (slot < po.cap) {
                            po.tgt[slot] = c;
                            po.key[slot] = kk;
                            atomicAdd(&po.per_tgt[c], 1);
                        } else {
                            atomicExch(po.err, 2);
                        }
                    }
                }
            }
        }
        auto key = [&](int idx) -> uint64_t { return pack_key(cd[idx], (uint32_t)cid[idx]); };
        // p's own list full (k distinct ids) and ordered by key: its k-th key
        // bounds the answer, so only the candidates below it can enter (few,
        // usually), and the new list is the merge of the two ordered runs.
        // Each output's rank is its position in its run plus the number of
        // keys of the other run below it (all keys are distinct).
        if (k <= 32 && nknown == k) {
            const uint64_t mk = lane < k ? key(lane) : kKeyMax;
            const uint64_t prev = __shfl_up_sync(KNNG_FULL_MASK, mk, 1);
            if (__all_sync(KNNG_FULL_MASK, lane == 0 || lane >= k || prev < mk)) {
                const uint64_t thr = __shfl_sync(KNNG_FULL_MASK, mk, k - 1);
                uint64_t* sv = keys + 64;  // the candidates below thr
                int ns = 0;
                for (int c0 = nknown; c0 < cnt; c0 += 32) {
                    const int i = c0 + lane;
                    const uint64_t kv = i < cnt ? key(i) : kKeyMax;
                    const bool below = kv < thr;
                    const uint32_t b = __ballot_sync(KNNG_FULL_MASK, below);
                    const int at = ns + __popc(b & lanemask_lt());
                    if (below && at < 32) sv[at] = kv;
                    ns += __popc(b);
                }
                if (ns <= 32) {
                    __syncwarp();
                    unsigned long long fl = 0;
                    const uint64_t x = lane < ns ? sv[lane] : kKeyMax;
                    int rx = 0, rm = lane;
                    for (int j = 0; j < ns; ++j) {
                        const uint64_t y = sv[j];
                        rx += y < x ? 1 : 0;
                        rm += y < mk ? 1 : 0;
                    }
                    if (lane < ns) {
                        int lo = 0, hi = k;  // own keys below x
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (key(mid) < x) lo = mid + 1;
                            else hi = mid;
                        }
                        rx += lo;
                        if (rx < k) {
                            ids_out[(int64_t)p * k + rx] = (int32_t)(uint32_t)x;
                            d_out[(int64_t)p * k + rx] = unord_key((uint32_t)(x >> 32));
                            fl |= 1ull << rx;
                        }
                    }
                    if (lane < k && rm < k) {
                        ids_out[(int64_t)p * k + rm] = (int32_t)(uint32_t)mk;
                        d_out[(int64_t)p * k + rm] = unord_key((uint32_t)(mk >> 32));
                    }
                    if (flags_out) {
#pragma unroll
                        for (int o = 16; o >= 1; o >>= 1) fl |= __shfl_xor_sync(KNNG_FULL_MASK, fl, o);
                        if (lane == 0) flags_out[p] = fl;
                    }
                    __syncwarp();
                    continue;
                }
            }
        }
        const int want = min(k, cnt);
        int nsel = 0;
        uint64_t v[E];
        if (cnt <= 512 && want <= 64) {
            nsel = cnt <= 256 ? warp_topk_sorted<8>(key, cnt, want, keys, keys + 64, hist)
                              : warp_topk_sorted<16>(key, cnt, want, keys, keys + 64, hist);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = lane * E + e;
                v[e] = i < nsel ? keys[i] : kKeyMax;
            }
        } else {
            if (want > 0) {
                const uint64_t thr = warp_select_threshold(key, cnt, want, hist);
                nsel = warp_compact_le(key, cnt, thr, sel);
            }
            __syncwarp();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int i = lane * E + e;
                v[e] = i < nsel ? key(sel[i]) : kKeyMax;
            }
            warp_bitonic_sort<E>(v);
        }
        int from[E];
        // new-entry flags: an output id is new unless it was in p's list
        unsigned long long fl = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = lane * E + e;
            from[e] = 0;
            if (i < nsel) {
                const int32_t id = (int32_t)(uint32_t)v[e];
                bool known = false;
                for (int q = 0; q < k; ++q) known |= (own[q] == id);
                from[e] = known ? 0 : 1;
            }
            if (i < k) {
                const bool ok = i < nsel;
                ids_out[(int64_t)p * k + i] = ok ? (int32_t)(uint32_t)v[e] : -1;
                d_out[(int64_t)p * k + i] = ok ? unord_key((uint32_t)(v[e] >> 32)) : __int_as_float(0x7f800000);
                if (from[e]) fl |= 1ull << i;
            }
        }
        if (flags_out) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) fl |= __shfl_xor_sync(KNNG_FULL_MASK, fl, o);
            if (lane == 0) flags_out[p] = fl;
        }
        __syncwarp();
    }
    if (stats) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) n_slots += __shfl_xor_sync(KNNG_FULL_MASK, n_slots, o);
        if (lane == 0) {
            atomicAdd(&stats[0], n_rows);
            atomicAdd(&stats[1], n_slots);
        }
    }
}

template <int E, int kDT>
static cudaError_t launch_prop(const XDesc& x, int k, const int32_t* order, const int32_t* ids_in, const float* d_in,
                               const unsigned long long* fin, int32_t* ids, float* dists, unsigned long long* fout,
                               const PairOffers& po, const uint8_t* tm, cudaStream_t st,
                               unsigned long long* stats)
{
    const PropLayout PL = prop_layout(k);
    int warps = (int)((200 * 1024) / PL.per_warp);
    if (warps > 8) warps = 8;
    if (warps < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = PL.per_warp * warps;
    // the build's first round (tree masks, no flags), a later first-order
    // round (flags), or the general form (pairwise offers, optional flags)
    const int mode = (tm && !fin && !po.tgt) ? 1 : (fin && !tm && !po.tgt) ? 2 : 0;
    auto kern = mode == 1 ? propagate_kernel<E, kDT, 1>
              : mode == 2 ? propagate_kernel<E, kDT, 2>
                          : propagate_kernel<E, kDT, 0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (int64_t)num_sms() * per_sm;
    const int64_t need = (x.n + warps - 1) / warps;
    if (blocks > need) blocks = need;
    RowLoader<kDT> rl{x.X, x.ld, x.d, x.vec};
    const RowLoader<kDtU8> rb{x.Xb, x.ldb, x.d, true};
    // byte rows scored one candidate per lane: 16-byte aligned rows whose
    // 16-byte blocks up to d stay inside the row (d <= 128)
    const uint8_t* lane_X = nullptr;
    int64_t lane_ld = 0;
    if (x.d <= 128) {
        if (kDT == kDtF32 && x.Xb) {
            lane_X = x.Xb;
            lane_ld = x.ldb;
        } else if (kDT == kDtU8 && (uintptr_t)x.X % 16 == 0 && x.ld % 16 == 0 && x.d % 16 == 0) {
            lane_X = static_cast<const uint8_t*>(x.X);
            lane_ld = x.ld;
        }
    }
    kern<<<(int)blocks, warps * 32, smem, st>>>(rl, rb, x.xb_bad, lane_X, lane_ld, po, x.n, k, order, ids_in, d_in, fin,
                                                tm, ids, dists, fout, PL.H, PL.hshift, PL.cap, (int)PL.per_warp,
                                                stats);
    note_launches(1);
    return cudaGetLastError();
}

template <int kDT>
static cudaError_t prop_dispatch(const XDesc& x, int k, const int32_t* order, const int32_t* ids_in,
                                 const float* d_in, const unsigned long long* fin, int32_t* ids, float* dists,
                                 unsigned long long* fout, const PairOffers& po, const uint8_t* tm,
                                 cudaStream_t st, unsigned long long* stats)
{
    if (k <= 32) return launch_prop<1, kDT>(x, k, order, ids_in, d_in, fin, ids, dists, fout, po, tm, st, stats);
    return launch_prop<2, kDT>(x, k, order, ids_in, d_in, fin, ids, dists, fout, po, tm, st, stats);
}

cudaError_t run_propagate(const XDesc& x, int k, const int32_t* order, const int32_t* ids_in, const float* d_in,
                          const unsigned long long* flags_in, int32_t* ids, float* dists,
                          unsigned long long* flags_out, cudaStream_t st, const PairOffers* offers,
                          const uint8_t* tmask_in, unsigned long long* stats)
{
    const PairOffers po = offers ? *offers : PairOffers{};
    if (x.dtype == kDtF16)
        return prop_dispatch<kDtF16>(x, k, order, ids_in, d_in, flags_in, ids, dists, flags_out, po, tmask_in, st,
                                     stats);
    if (x.dtype == kDtU8)
        return prop_dispatch<kDtU8>(x, k, order, ids_in, d_in, flags_in, ids, dists, flags_out, po, tmask_in, st,
                                    stats);
    return prop_dispatch<kDtF32>(x, k, order, ids_in, d_in, flags_in, ids, dists, flags_out, po, tmask_in, st, stats);
}

}  // namespace knng
