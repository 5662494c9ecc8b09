// Exact k-NN lists (Def. 1 of arXiv:1307.7852) of a set of query points
// against all n points, by brute force with the canonical FP32 distance.
// This is the yardstick of the accuracy measure of Sec. 4 (recall on a
// sample of points), not part of the approximate method.
//
// One block of QB warps serves QB queries; candidate rows stream through
// shared memory in tiles of 32 rows, so each row is read once per block.
// Every warp keeps a buffer of keys below its current k-th best and shrinks
// it to the k best (warp radix select) whenever it fills.
#include <type_traits>

#include "knng_common.cuh"
#include "knng_internal.h"

namespace knng {

namespace {
constexpr int kQB = 8;  // queries (warps) per block
}

template <int kDT>
__global__ void __launch_bounds__(kQB * 32) exact_knn_kernel(RowLoader<kDT> L, int64_t n,
                                                             const int32_t* __restrict__ queries, int nq,
                                                             int k, int cap, int32_t* __restrict__ out_ids,
                                                             float* __restrict__ out_d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int dp = (L.d + 3) & ~3;
    // shared memory: tile[32][dp] | qrow[kQB][dp] | buf[kQB][cap] | hist[kQB][256] | sel[kQB][64]
    float* tile = reinterpret_cast<float*>(smem_raw);
    float* qrow = tile + 32 * dp;
    unsigned long long* buf_all = reinterpret_cast<unsigned long long*>(qrow + kQB * dp);
    uint32_t* hist_all = reinterpret_cast<uint32_t*>(buf_all + (size_t)kQB * cap);
    int* sel_all = reinterpret_cast<int*>(hist_all + 256 * kQB);
    unsigned long long* buf = buf_all + (size_t)w * cap;
    uint32_t* hist = hist_all + 256 * w;
    int* sel = sel_all + 64 * w;

    const int qi = blockIdx.x * kQB + w;
    const int32_t qraw = qi < nq ? queries[qi] : 0;
    const bool valid = qraw >= 0 && qraw < n;  // an out-of-range query gets an empty row
    const bool active = qi < nq && valid;
    const int32_t q = valid ? qraw : 0;
    for (int j = 4 * lane; j < dp; j += 128) {
        const float4 v = L.load4(q, j);
        *reinterpret_cast<float4*>(qrow + w * dp + j) = v;
    }
    unsigned long long thr = kKeyMax;
    int nb = 0;
    for (int64_t j0 = 0; j0 < n; j0 += 32) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < 32 * (dp / 4); idx += kQB * 32) {
            const int r = idx / (dp / 4), c = 4 * (idx % (dp / 4));
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j0 + r < n) v = L.load4(j0 + r, c);
            *reinterpret_cast<float4*>(tile + r * dp + c) = v;
        }
        __syncthreads();
        if (!active) continue;
        unsigned long long mine = kKeyMax;
        const int rows = (n - j0) < 32 ? (int)(n - j0) : 32;
        for (int r = 0; r < rows; ++r) {
            // the canonical distance (blocks of 32 entries added in order)
            float tot = 0.f;
            for (int c0 = 0; c0 < L.d; c0 += 128) {
                const int j = c0 + 4 * lane;
                float s = 0.f;
                if (j < dp) {
                    const float4 a = *reinterpret_cast<const float4*>(qrow + w * dp + j);
                    const float4 b = *reinterpret_cast<const float4*>(tile + r * dp + j);
                    float t;
                    t = a.x - b.x; s = fmaf(t, t, s);
                    t = a.y - b.y; s = fmaf(t, t, s);
                    t = a.z - b.z; s = fmaf(t, t, s);
                    t = a.w - b.w; s = fmaf(t, t, s);
                }
                s += __shfl_xor_sync(KNNG_FULL_MASK, s, 4);
                s += __shfl_xor_sync(KNNG_FULL_MASK, s, 2);
                s += __shfl_xor_sync(KNNG_FULL_MASK, s, 1);
                tot = chunk_blocks_add(tot, s);
            }
            if (lane == r && j0 + r != q) mine = pack_key(tot, (uint32_t)(j0 + r));
        }
        const bool take = mine < thr;
        const uint32_t b = __ballot_sync(KNNG_FULL_MASK, take);
        if (take) buf[nb + __popc(b & lanemask_lt())] = mine;
        nb += __popc(b);
        if (nb > cap - 32) {
            __syncwarp();
            auto key = [&](int i) -> uint64_t { return buf[i]; };
            const uint64_t t2 = warp_select_threshold(key, nb, k, hist);
            const int m = warp_compact_le(key, nb, t2, sel);
            __syncwarp();
            unsigned long long keep0 = lane < m ? buf[sel[lane]] : kKeyMax;
            unsigned long long keep1 = lane + 32 < m ? buf[sel[lane + 32]] : kKeyMax;
            __syncwarp();
            if (lane < m) buf[lane] = keep0;
            if (lane + 32 < m) buf[lane + 32] = keep1;
            nb = m;
            thr = t2;
            __syncwarp();
        }
    }
    if (qi >= nq) return;
    if (!valid) nb = 0;
    __syncwarp();
    auto key = [&](int i) -> uint64_t { return buf[i]; };
    const int want = min(k, nb);
    int m = 0;
    if (want > 0) {
        const uint64_t t2 = warp_select_threshold(key, nb, want, hist);
        m = warp_compact_le(key, nb, t2, sel);
    }
    __syncwarp();
    uint64_t v[2];
    v[0] = 2 * lane < m ? buf[sel[2 * lane]] : kKeyMax;
    v[1] = 2 * lane + 1 < m ? buf[sel[2 * lane + 1]] : kKeyMax;
    warp_bitonic_sort<2>(v);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int i = 2 * lane + e;
        if (i < k) {
            const bool ok = i < m;
            out_ids[(int64_t)qi * k + i] = ok ? (int32_t)(uint32_t)v[e] : -1;
            out_d[(int64_t)qi * k + i] = ok ? unord_key((uint32_t)(v[e] >> 32)) : __int_as_float(0x7f800000);
        }
    }
}

cudaError_t run_exact_knn(const XDesc& x, const int32_t* queries, int nq, int k, int32_t* ids,
                          float* dists, cudaStream_t st)
{
    const int dp = (x.d + 3) & ~3;
    const int cap = 4 * k + 64;
    const size_t smem = sizeof(float) * (size_t)(32 + kQB) * dp + sizeof(unsigned long long) * (size_t)kQB * cap +
                        sizeof(uint32_t) * 256 * kQB + sizeof(int) * 64 * kQB;
    if (smem > 220 * 1024) return cudaErrorInvalidConfiguration;
    const int grid = (nq + kQB - 1) / kQB;
    auto launch = [&](auto dt) {
        constexpr int kDT = decltype(dt)::value;
        auto kern = exact_knn_kernel<kDT>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        RowLoader<kDT> rl{x.X, x.ld, x.d, x.vec};
        kern<<<grid, kQB * 32, smem, st>>>(rl, x.n, queries, nq, k, cap, ids, dists);
        note_launches(1);
    };
    if (x.dtype == kDtF16) launch(std::integral_constant<int, kDtF16>{});
    else if (x.dtype == kDtU8) launch(std::integral_constant<int, kDtU8>{});
    else launch(std::integral_constant<int, kDtF32>{});
    return cudaGetLastError();
}

}  // namespace knng
