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

}  // namespace knng
