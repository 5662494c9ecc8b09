// Combination of the T base graphs (Sec. 3.1 of arXiv:1307.7852): every
// point unites its T adjacency lists and keeps the k nearest.
//
// A group of GS lanes per point (GS the power of two >= T), lane j walking
// tree j's row.  The T input rows are each ordered by (dist, id), so a T-way
// merge on the packed 64-bit key (ord(dist) << 32 | id) visits the union in
// output order: every step takes the group minimum of the lanes' heads and
// advances the lanes holding it (the same neighbour found by several trees
// has equal keys, so its copies go together); a neighbour seen again with
// a different distance is dropped by the id check against the entries
// already taken, and p itself is skipped.  A warp's rows (32 / GS points,
// contiguous for every tree) are staged in shared memory; output slot s of a
// point is held by lane s % GS of its group.
// With eight lanes a group also records, per output entry, the trees whose
// rows held it (the lanes that advanced on it).
#include "knng_common.cuh"
#include "knng_internal.h"

namespace knng {

constexpr int kMergeThreads = 128;

// Staging: the ids and distances of a warp's rows land in shared memory by
// 4-byte cp.async copies, all of a batch in flight at once.
template <int GS, int R>
__global__ void __launch_bounds__(kMergeThreads) merge_kernel(int64_t n, int T, int k,
                                                              const int32_t* __restrict__ ids_in,
                                                              const float* __restrict__ d_in,
                                                              int32_t* __restrict__ ids, float* __restrict__ dists,
                                                              uint8_t* __restrict__ tmask,
                                                              const int* __restrict__ all_exact)
{
    constexpr int PPW = 32 / GS;  // points per warp
    constexpr int NW = kMergeThreads / 32;
    extern __shared__ __align__(16) int32_t mraw[];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int grp = lane / GS, j = lane % GS;
    const int ks = k | 1;  // odd row stride: a group's lanes read rows in different banks
    const int buf_words = 2 * 32 * ks;  // ids [PPW][GS][ks], then distances
    int32_t* wbuf = mraw + (size_t)wq * buf_words;
    const unsigned gmask = GS == 32 ? 0xFFFFFFFFu : (((1u << GS) - 1u) << (grp * GS));
    const int64_t step = (int64_t)gridDim.x * NW * PPW;
    // tree masks (GS == 8) only when every leaf list was exact
    const bool masks = GS == 8 && tmask && all_exact && *all_exact != 0;
    const int dpp = 32 / k, dh = 32 - (32 / k) * k;
    // for every tree the rows of a batch's points are contiguous; entry
    // e = pp k + h of them, advanced by 32 without division
    auto stage = [&](int64_t wbase) {
        int32_t* sid = wbuf;
        float* sd = reinterpret_cast<float*>(sid + 32 * ks);
        const int np = (int)(n - wbase < PPW ? n - wbase : PPW);
        for (int t = 0; t < T; ++t) {
            const int64_t src = ((int64_t)t * n + wbase) * k;
            int pp = lane / k, h = lane - (lane / k) * k;
            for (int e = lane; e < np * k; e += 32) {
                const int o = (pp * GS + t) * ks + h;
                cp_async4(sid + o, ids_in + src + e);
                cp_async4(sd + o, d_in + src + e);
                pp += dpp;
                h += dh;
                if (h >= k) {
                    h -= k;
                    ++pp;
                }
            }
        }
    };
    for (int64_t wbase = ((int64_t)blockIdx.x * NW + wq) * PPW; wbase < n; wbase += step) {
        stage(wbase);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
        const int np = (int)(n - wbase < PPW ? n - wbase : PPW);
        const int64_t p = wbase + grp;
        const bool live = grp < np;
        const int32_t* rid = wbuf + (grp * GS + j) * ks;
        const float* rd = reinterpret_cast<const float*>(wbuf + 32 * ks) + (grp * GS + j) * ks;
        auto row = [&](int h) -> unsigned long long {
            const int32_t id = rid[h];
            return id >= 0 ? pack_key(rd[h], (uint32_t)id) : kKeyMax;
        };
        int h = 0;
        // a row ends at its first empty entry (kKeyMax); trees j >= T are empty
        unsigned long long key = (live && j < T) ? row(0) : kKeyMax;
        unsigned long long o[R];
        uint32_t om[R];  // trees of the held entries
#pragma unroll
        for (int r = 0; r < R; ++r) {
            o[r] = kKeyMax;
            om[r] = 0u;
        }
        int cnt = 0;
        // ids taken so far, as one bit of a 64-bit filter (the same in every
        // lane of the group): the full id check runs only on a hit
        unsigned long long taken = 0ull;
        bool done = !live || k == 0;
        while (__any_sync(KNNG_FULL_MASK, !done)) {
            unsigned long long best = key;
#pragma unroll
            for (int off = GS / 2; off >= 1; off >>= 1) {
                const unsigned long long other = __shfl_xor_sync(KNNG_FULL_MASK, best, off, GS);
                best = other < best ? other : best;
            }
            if (!done) {  // uniform over the group
                if (best == kKeyMax) {
                    done = true;
                } else {
                    const bool hit = key == best;
                    uint32_t trees = 0u;
                    if constexpr (GS == 8) trees = (__ballot_sync(gmask, hit) >> (grp * GS)) & 0xFFu;
                    if (hit) {
                        ++h;
                        key = h < k ? row(h) : kKeyMax;
                    }
                    const int32_t id = (int32_t)(uint32_t)best;
                    const unsigned long long bit = 1ull << (((uint32_t)id * 0x9E3779B1u) >> 26);
                    bool dup = id == (int32_t)p;
                    if (!dup && (taken & bit)) {
#pragma unroll
                        for (int r = 0; r < R; ++r) dup |= (GS * r + j < cnt) && ((int32_t)(uint32_t)o[r] == id);
                        dup = __any_sync(gmask, dup);
                    }
                    if (!dup) {
#pragma unroll
                        for (int r = 0; r < R; ++r)
                            if (GS * r + j == cnt) {
                                o[r] = best;
                                om[r] = trees;
                            }
                        taken |= bit;
                        ++cnt;
                        done = cnt == k;
                    }
                }
            }
        }
        if (live) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int s2 = GS * r + j;
                if (s2 < k) {
                    const bool ok = s2 < cnt;
                    ids[p * k + s2] = ok ? (int32_t)(uint32_t)o[r] : -1;
                    dists[p * k + s2] = ok ? unord_key((uint32_t)(o[r] >> 32)) : __int_as_float(0x7f800000);
                    if (GS == 8 && tmask) tmask[p * k + s2] = (ok && masks) ? (uint8_t)om[r] : (uint8_t)0;
                }
            }
        }
        __syncwarp();  // the rows are read before the next batch lands
    }
}

template <int GS, int R>
static cudaError_t launch_merge(int64_t n, int T, int k, const int32_t* ids_in, const float* d_in, int32_t* ids,
                                float* dists, uint8_t* tmask, const int* all_exact, cudaStream_t st)
{
    static bool attr = false;  // one per instantiation
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(merge_kernel<GS, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((kMergeThreads / 32) * 2 * 32 * (kMaxK | 1) * sizeof(int32_t)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const size_t smem = (size_t)(kMergeThreads / 32) * 2 * 32 * (k | 1) * sizeof(int32_t);
    const int64_t per_block = (int64_t)(kMergeThreads / 32) * (32 / GS);
    const int64_t want = (n + per_block - 1) / per_block;
    // resident blocks only: each warp then merges many batches, with the
    // next batch's copies in flight
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, merge_kernel<GS, R>, kMergeThreads, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t resident = (int64_t)num_sms() * per_sm;
    const int grid = (int)(want < resident ? want : resident);
    merge_kernel<GS, R><<<grid, kMergeThreads, smem, st>>>(n, T, k, ids_in, d_in, ids, dists, tmask, all_exact);
    return cudaSuccess;
}

cudaError_t run_merge(int64_t n, int T, int k, const int32_t* ids_in, const float* d_in,
                      int32_t* ids, float* dists, cudaStream_t st, uint8_t* tmask, const int* all_exact)
{
    cudaError_t e;
    if (T <= 8) e = k <= 32 ? launch_merge<8, 4>(n, T, k, ids_in, d_in, ids, dists, tmask, all_exact, st)
                            : launch_merge<8, 8>(n, T, k, ids_in, d_in, ids, dists, tmask, all_exact, st);
    else if (T <= 16) e = launch_merge<16, 4>(n, T, k, ids_in, d_in, ids, dists, nullptr, nullptr, st);
    else e = launch_merge<32, 2>(n, T, k, ids_in, d_in, ids, dists, nullptr, nullptr, st);
    if (e != cudaSuccess) return e;
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adding one division to the running graph (Sec. 3.2's effective rate): the
// k best of the running list a and the new tree's list b, and the count of
// output entries that were not in a (counts[0]) and of all output entries
// (counts[1]), summed over the points: r_m = counts[0] / counts[1].
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) merge_add_kernel(int64_t n, int k, const int32_t* __restrict__ ia,
                                                        const float* __restrict__ da, const int32_t* __restrict__ ib,
                                                        const float* __restrict__ db, int32_t* __restrict__ ids,
                                                        float* __restrict__ dists,
                                                        unsigned long long* __restrict__ counts)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned long long nnew = 0, ntot = 0;
    if (p < n) {
        const int32_t* la = ia + p * k;
        const int32_t* lb = ib + p * k;
        const float* fa = da + p * k;
        const float* fb = db + p * k;
        auto key_of = [&](const int32_t* l, const float* f, int h) -> uint64_t {
            if (h >= k || l[h] < 0) return kKeyMax;
            return pack_key(f[h], (uint32_t)l[h]);
        };
        int ha = 0, hb = 0, cnt = 0;
        uint64_t ka = key_of(la, fa, 0), kb = key_of(lb, fb, 0);
        int32_t* oi = ids + p * k;
        float* od = dists + p * k;
        while (cnt < k) {
            const uint64_t best = ka < kb ? ka : kb;
            if (best == kKeyMax) break;
            const bool from_a = ka == best;
            if (ka == best) ka = key_of(la, fa, ++ha);
            if (kb == best) kb = key_of(lb, fb, ++hb);
            const int32_t id = (int32_t)(uint32_t)best;
            if (id == (int32_t)p) continue;
            bool dup = false;
            for (int e = 0; e < cnt; ++e) dup |= (oi[e] == id);
            if (dup) continue;
            bool in_a = from_a;
            for (int e = 0; e < k && !in_a; ++e) in_a = la[e] == id;
            nnew += in_a ? 0 : 1;
            oi[cnt] = id;
            od[cnt] = unord_key((uint32_t)(best >> 32));
            ++cnt;
        }
        ntot = (unsigned long long)cnt;
        for (int e = cnt; e < k; ++e) {
            oi[e] = -1;
            od[e] = __int_as_float(0x7f800000);
        }
    }
    // block sums, one atomic pair per block
    for (int o = 16; o >= 1; o >>= 1) {
        nnew += __shfl_xor_sync(KNNG_FULL_MASK, nnew, o);
        ntot += __shfl_xor_sync(KNNG_FULL_MASK, ntot, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counts[0], nnew);
        atomicAdd(&counts[1], ntot);
    }
}

cudaError_t run_merge_add(int64_t n, int k, const int32_t* ia, const float* da, const int32_t* ib, const float* db,
                          int32_t* ids, float* dists, unsigned long long* counts, cudaStream_t st)
{
    const int grid = (int)((n + 127) / 128);
    merge_add_kernel<<<grid, 128, 0, st>>>(n, k, ia, da, ib, db, ids, dists, counts);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace knng
