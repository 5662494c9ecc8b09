// Pairwise updating (Sec. 3.4 of arXiv:1307.7852: when v is considered for
// u's list, u is also considered for v's list) in a synchronous
// first-order round.  With C(p) = N(p) u N(N(p)) \ {p}, the new list of p is
// the k best of C(p) and of every q with p in C(q).
//  1. The forward kernel (propagate.cu) builds every point's own k best of
//     C(p) and offers (c, (D, p)) for every c in C(p) whose input list p
//     would enter -- (D, p) below c's k-th input (dist, id); any other offer
//     cannot reach c's new list, which is never worse than its input list.
//     Pairs skipped as scored in the previous round were offered then.
//  2. The offers are grouped by target: per-target counts (taken during
//     emission), an exclusive scan, a scatter.
//  3. One warp per point merges its forward list with its offers (equal
//     keys are the same neighbour) and keeps the k best; the new-entry flags
//     mark the ids that were not in the point's input list.
#include "knng_common.cuh"
#include "knng_internal.h"

namespace knng {

namespace {
constexpr int kScanTile = 4096;  // counts per scan block (1024 threads x 4)
}

void pairwise_take(Arena& a, int64_t n, int k, PairScratch& s)
{
    // capacity: four offers per list entry (overflow sets the error word)
    const unsigned long long cap = (unsigned long long)n * k * 4;
    s.po.cap = cap;
    s.po.tgt = a.take<int32_t>(cap);
    s.po.key = a.take<uint64_t>(cap);
    s.po.count = a.take<unsigned long long>(1);
    s.po.per_tgt = a.take<int32_t>((size_t)n);
    s.off = a.take<int64_t>((size_t)n + 1);
    s.bsum = a.take<int64_t>((size_t)(n + kScanTile - 1) / kScanTile + 1);
    s.sorted = a.take<uint64_t>(cap);
    s.fwd_i = a.take<int32_t>((size_t)n * k);
    s.fwd_d = a.take<float>((size_t)n * k);
}

// ---- exclusive scan of the per-target counts -----------------------------
__device__ __forceinline__ int64_t block_incl_scan(int64_t v, int64_t* wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(KNNG_FULL_MASK, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        int64_t x = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(KNNG_FULL_MASK, x, o);
            if (lane >= o) x += t;
        }
        wsum[lane] = x;
    }
    __syncthreads();
    const int64_t r = v + (w > 0 ? wsum[w - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) scan_tiles_kernel(const int32_t* __restrict__ cnt, int64_t n,
                                                          int64_t* __restrict__ bsum)
{
    __shared__ int64_t wsum[32];
    const int64_t b0 = (int64_t)blockIdx.x * kScanTile;
    int64_t v = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t i = b0 + threadIdx.x * 4 + e;
        if (i < n) v += cnt[i];
    }
    const int64_t inc = block_incl_scan(v, wsum);
    if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = inc;
}

// one block: exclusive scan of the nb tile sums in place, total to bsum[nb]
__global__ void __launch_bounds__(1024) scan_sums_kernel(int64_t* __restrict__ bsum, int64_t nb)
{
    __shared__ int64_t wsum[32];
    int64_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
        const int64_t i = c0 + threadIdx.x;
        const int64_t v = i < nb ? bsum[i] : 0;
        const int64_t inc = block_incl_scan(v, wsum);
        if (i < nb) bsum[i] = carry + inc - v;
        __shared__ int64_t last;
        if (threadIdx.x == 1023) last = inc;
        __syncthreads();
        carry += last;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

__global__ void __launch_bounds__(1024) scan_apply_kernel(const int32_t* __restrict__ cnt, int64_t n,
                                                          const int64_t* __restrict__ bsum, int64_t nb,
                                                          int64_t* __restrict__ off)
{
    __shared__ int64_t wsum[32];
    const int64_t b0 = (int64_t)blockIdx.x * kScanTile;
    int64_t c[4];
    int64_t v = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t i = b0 + threadIdx.x * 4 + e;
        c[e] = i < n ? cnt[i] : 0;
        v += c[e];
    }
    int64_t run = block_incl_scan(v, wsum) - v + bsum[blockIdx.x];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t i = b0 + threadIdx.x * 4 + e;
        if (i < n) off[i] = run;
        run += c[e];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[n] = bsum[nb];
}

// offers into their target's bucket; per_tgt counts back to zero
__global__ void scatter_offers_kernel(PairOffers po, const int64_t* __restrict__ off, uint64_t* __restrict__ sorted)
{
    const unsigned long long total = *po.count < po.cap ? *po.count : po.cap;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < total;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t c = po.tgt[i];
        const int slot = atomicSub(&po.per_tgt[c], 1) - 1;
        sorted[off[c] + slot] = po.key[i];
    }
}

// ---- per point: forward list + offers -> k best ---------------------------
__global__ void __launch_bounds__(256) pair_merge_kernel(int64_t n, int k, const int32_t* __restrict__ ids_in,
                                                         const int32_t* __restrict__ fwd_i,
                                                         const float* __restrict__ fwd_d,
                                                         const int64_t* __restrict__ off,
                                                         const uint64_t* __restrict__ sorted,
                                                         int32_t* __restrict__ ids, float* __restrict__ dists,
                                                         unsigned long long* __restrict__ flags_out)
{
    __shared__ uint64_t cur_all[8][128];
    __shared__ int32_t own_all[8][64];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t* cur = cur_all[w];
    int32_t* own = own_all[w];
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = gw; p < n; p += nw) {
        // the forward list, as keys, in slots [0, 64)
        for (int i = lane; i < 64; i += 32) {
            uint64_t v = kKeyMax;
            if (i < k) {
                const int32_t id = fwd_i[p * k + i];
                if (id >= 0) v = pack_key(fwd_d[p * k + i], (uint32_t)id);
                own[i] = ids_in[p * k + i];
            }
            cur[i] = v;
        }
        __syncwarp();
        const int64_t o0 = off[p], o1 = off[p + 1];
        for (int64_t c0 = o0; c0 < o1; c0 += 64) {
            // next 64 offers in slots [64, 128), the ones already held dropped
            for (int i = lane; i < 64; i += 32) {
                uint64_t v = kKeyMax;
                if (c0 + i < o1) {
                    v = sorted[c0 + i];
                    for (int j = 0; j < k; ++j)
                        if (cur[j] == v) v = kKeyMax;
                }
                cur[64 + i] = v;
            }
            __syncwarp();
            uint64_t v4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v4[e] = cur[lane * 4 + e];
            __syncwarp();
            warp_bitonic_sort<4>(v4);
#pragma unroll
            for (int e = 0; e < 4; ++e) cur[lane * 4 + e] = v4[e];
            __syncwarp();
        }
        unsigned long long fl = 0;
        for (int i = lane; i < k; i += 32) {
            const uint64_t v = cur[i];
            const bool ok = v != kKeyMax;
            const int32_t id = ok ? (int32_t)(uint32_t)v : -1;
            ids[p * k + i] = id;
            dists[p * k + i] = ok ? unord_key((uint32_t)(v >> 32)) : __int_as_float(0x7f800000);
            bool known = false;
            for (int q = 0; q < k; ++q) known |= (own[q] == id);
            if (ok && !known) fl |= 1ull << i;
        }
        if (flags_out) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) fl |= __shfl_xor_sync(KNNG_FULL_MASK, fl, o);
            if (lane == 0) flags_out[p] = fl;
        }
        __syncwarp();
    }
}

cudaError_t run_propagate_pairwise(const XDesc& x, int k, const int32_t* order, const int32_t* ids_in,
                                   const float* d_in, const unsigned long long* flags_in, int32_t* ids, float* dists,
                                   unsigned long long* flags_out, const PairScratch& s, int* err, cudaStream_t st)
{
    const int64_t n = x.n;
    PairOffers po = s.po;
    po.err = err;
    cudaError_t e = cudaMemsetAsync(po.count, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(po.per_tgt, 0, sizeof(int32_t) * (size_t)n, st);
    if (e != cudaSuccess) return e;
    // 1. forward lists and offers
    e = run_propagate(x, k, order, ids_in, d_in, flags_in, s.fwd_i, s.fwd_d, nullptr, st, &po);
    if (e != cudaSuccess) return e;
    // 2. group the offers by target
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    scan_tiles_kernel<<<(unsigned)nb, 1024, 0, st>>>(po.per_tgt, n, s.bsum);
    scan_sums_kernel<<<1, 1024, 0, st>>>(s.bsum, nb);
    scan_apply_kernel<<<(unsigned)nb, 1024, 0, st>>>(po.per_tgt, n, s.bsum, nb, s.off);
    scatter_offers_kernel<<<num_sms() * 8, 256, 0, st>>>(po, s.off, s.sorted);
    note_launches(4);
    // 3. merge
    const int grid = (int)std::min<int64_t>((n + 7) / 8, (int64_t)num_sms() * 16);
    pair_merge_kernel<<<grid, 256, 0, st>>>(n, k, ids_in, s.fwd_i, s.fwd_d, s.off, s.sorted, ids, dists, flags_out);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace knng
