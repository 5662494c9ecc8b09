// Combination of the T base graphs (Sec. 3.1 of arXiv:1307.7852): every
// point unites its T adjacency lists and keeps the k nearest.
//
// One thread per point.  The T input rows are each ordered by (dist, id),
// so a T-way merge on the packed 64-bit key (ord(dist) << 32 | id) visits the
// union in output order; equal keys (the same neighbour found by several
// trees) advance together, and a neighbour seen again with a different
// distance is dropped by the id check against the rows already written.
#include "knng_common.cuh"
#include "knng_internal.h"

namespace knng {

template <int TMAX>
__global__ void __launch_bounds__(128) merge_kernel(int64_t n, int T, int k,
                                                    const int32_t* __restrict__ ids_in,
                                                    const float* __restrict__ d_in,
                                                    int32_t* __restrict__ ids, float* __restrict__ dists)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int h[TMAX];
    uint64_t cur[TMAX];
#pragma unroll
    for (int t = 0; t < TMAX; ++t) {
        h[t] = 0;
        cur[t] = kKeyMax;
        if (t < T) {
            const int64_t r = ((int64_t)t * n + p) * k;
            const int32_t id = ids_in[r];
            if (id >= 0) cur[t] = pack_key(d_in[r], (uint32_t)id);
        }
    }
    int32_t* oi = ids + p * k;
    float* od = dists + p * k;
    int cnt = 0;
    while (cnt < k) {
        uint64_t best = kKeyMax;
#pragma unroll
        for (int t = 0; t < TMAX; ++t) best = cur[t] < best ? cur[t] : best;
        if (best == kKeyMax) break;
#pragma unroll
        for (int t = 0; t < TMAX; ++t) {
            if (cur[t] == best) {
                ++h[t];
                cur[t] = kKeyMax;
                if (h[t] < k) {
                    const int64_t r = ((int64_t)t * n + p) * k + h[t];
                    const int32_t id = ids_in[r];
                    if (id >= 0) cur[t] = pack_key(d_in[r], (uint32_t)id);
                }
            }
        }
        const int32_t id = (int32_t)(uint32_t)best;
        if (id == (int32_t)p) continue;
        bool dup = false;
        for (int e = 0; e < cnt; ++e) dup |= (oi[e] == id);
        if (dup) continue;
        oi[cnt] = id;
        od[cnt] = unord_key((uint32_t)(best >> 32));
        ++cnt;
    }
    for (int e = cnt; e < k; ++e) {
        oi[e] = -1;
        od[e] = __int_as_float(0x7f800000);
    }
}

cudaError_t run_merge(int64_t n, int T, int k, const int32_t* ids_in, const float* d_in,
                      int32_t* ids, float* dists, cudaStream_t st)
{
    const int grid = (int)((n + 127) / 128);
    if (T <= 4) merge_kernel<4><<<grid, 128, 0, st>>>(n, T, k, ids_in, d_in, ids, dists);
    else if (T <= 8) merge_kernel<8><<<grid, 128, 0, st>>>(n, T, k, ids_in, d_in, ids, dists);
    else if (T <= 16) merge_kernel<16><<<grid, 128, 0, st>>>(n, T, k, ids_in, d_in, ids, dists);
    else merge_kernel<32><<<grid, 128, 0, st>>>(n, T, k, ids_in, d_in, ids, dists);
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
