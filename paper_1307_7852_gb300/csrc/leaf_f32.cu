// Leaf graphs, FP32 candidate stage (Sec. 3.1 of arXiv:1307.7852: a brute-
// force k-NN graph inside every leaf subset).
//
// One block per (leaf, tree).  For every block of 32 rows of the leaf:
//   1. Gram S = X_rows X_leaf^T in FP32 SIMT (register-tiled, K in slices of
//      32 staged transposed in shared memory), D~ = |x|^2 + |y|^2 - 2 S;
//   2. one warp per row picks the k' smallest (D~, id) by radix select;
//   3. the k' candidates are rescored by the canonical FP32 direct-difference
//      distance and sorted; the k best are written.
// Leaf members are in ascending id order, so a local index ranks like the id.
#include <algorithm>

#include "knng_common.cuh"
#include "knng_internal.h"

namespace knng {

namespace {
constexpr int kRB = 32;   // rows per block pass
constexpr int kKC = 32;   // K slice
constexpr int kNT = 256;  // threads
constexpr int kCandCap = 128;

struct LeafSmem {
    int32_t* lid;
    float* nrm;
    float* Bt;
    float* D;
    unsigned char* ws;  // kLeafWarpScratch per warp
};

__host__ __device__ inline size_t leaf_smem_bytes(int m_pad)
{
    return sizeof(int32_t) * m_pad + sizeof(float) * m_pad + sizeof(float) * kKC * (m_pad + 1) +
           sizeof(float) * kRB * m_pad + 16 + (kNT / 32) * kLeafWarpScratch;
}
}  // namespace

template <int CT, int kDT>
__global__ void __launch_bounds__(kNT) leaf_knn_f32_kernel(RowLoader<kDT> L, int64_t n,
                                                           const int32_t* __restrict__ perm,
                                                           const int32_t* __restrict__ leaf_off, int k,
                                                           int kp, int32_t* __restrict__ out_ids,
                                                           float* __restrict__ out_d)
{
    constexpr int m_pad = 32 * CT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LeafSmem sm;
    {
        unsigned char* p = smem_raw;
        sm.lid = reinterpret_cast<int32_t*>(p); p += sizeof(int32_t) * m_pad;
        sm.nrm = reinterpret_cast<float*>(p); p += sizeof(float) * m_pad;
        sm.Bt = reinterpret_cast<float*>(p); p += sizeof(float) * kKC * (m_pad + 1);
        sm.D = reinterpret_cast<float*>(p); p += sizeof(float) * kRB * m_pad;
        sm.ws = reinterpret_cast<unsigned char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    }
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int tx = tid & 31, ty = tid >> 5;
    const int t = blockIdx.y;
    const int b = leaf_off[blockIdx.x];
    const int m = leaf_off[blockIdx.x + 1] - b;
    const int32_t* prow = perm + (int64_t)t * n + b;
    for (int j = tid; j < m_pad; j += kNT) {
        sm.lid[j] = j < m ? prow[j] : -1;
        sm.nrm[j] = 0.f;
    }
    __syncthreads();
    // squared norms (any order: they only feed the candidate distances)
    for (int r = w; r < m; r += kNT / 32) {
        float s = 0.f;
        for (int j = 4 * lane; j < L.d; j += 128) {
            const float4 x = L.load4(sm.lid[r], j);
            s = fmaf(x.x, x.x, s); s = fmaf(x.y, x.y, s); s = fmaf(x.z, x.z, s); s = fmaf(x.w, x.w, s);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(KNNG_FULL_MASK, s, o);
        if (lane == 0) sm.nrm[r] = s;
    }
    unsigned char* ws = sm.ws + (size_t)kLeafWarpScratch * w;
    constexpr int mp1 = m_pad + 1;

    for (int rb = 0; rb < m; rb += kRB) {
        float acc[4][CT];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int c = 0; c < CT; ++c) acc[rr][c] = 0.f;
        for (int k0 = 0; k0 < L.d; k0 += kKC) {
            __syncthreads();
            // four entries a load (zero past d), stored transposed
            for (int idx = tid; idx < m_pad * (kKC / 4); idx += kNT) {
                const int row = idx / (kKC / 4), kk = 4 * (idx % (kKC / 4));
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (row < m && k0 + kk < L.d) v = L.load4(sm.lid[row], k0 + kk);
                sm.Bt[(kk + 0) * mp1 + row] = v.x;
                sm.Bt[(kk + 1) * mp1 + row] = v.y;
                sm.Bt[(kk + 2) * mp1 + row] = v.z;
                sm.Bt[(kk + 3) * mp1 + row] = v.w;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < kKC; ++kk) {
                float a[4], bb[CT];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) a[rr] = sm.Bt[kk * mp1 + rb + ty * 4 + rr];
#pragma unroll
                for (int c = 0; c < CT; ++c) bb[c] = sm.Bt[kk * mp1 + tx + 32 * c];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                    for (int c = 0; c < CT; ++c) acc[rr][c] = fmaf(a[rr], bb[c], acc[rr][c]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int r = ty * 4 + rr;
            const float ni = sm.nrm[min(rb + r, m_pad - 1)];
#pragma unroll
            for (int c = 0; c < CT; ++c) {
                const int col = tx + 32 * c;
                sm.D[r * m_pad + col] = ni + sm.nrm[col] - 2.f * acc[rr][c];
            }
        }
        __syncthreads();
        for (int r = w; r < kRB; r += kNT / 32) {
            const int row = rb + r;
            if (row >= m) break;
            const float* Drow = sm.D + r * m_pad;
            const int gi = sm.lid[row];
            leaf_row_finish<CT, kDT>(L, [&](int j) { return Drow[j]; }, m, row, sm.lid, k, kp, ws,
                                  out_ids + ((int64_t)t * n + gi) * k, out_d + ((int64_t)t * n + gi) * k);
        }
    }
}

template <int CT, int kDT>
static cudaError_t launch_leaf_f32(const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                                   const int32_t* perm, int k, int kp, int32_t* ids, float* dists,
                                   cudaStream_t st)
{
    const size_t smem = leaf_smem_bytes(32 * CT);
    auto kern = leaf_knn_f32_kernel<CT, kDT>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)leaf_smem_bytes(32 * CT));
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    RowLoader<kDT> rl{x.X, x.ld, x.d, x.vec};
    const int nleaves = (int)P.leaf_off.size() - 1;
    kern<<<dim3(nleaves, T), kNT, smem, st>>>(rl, x.n, perm, dp.leaf_off, k, kp, ids, dists);
    note_launches(1);
    return cudaGetLastError();
}

template <int kDT>
static cudaError_t dispatch_ct(const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                               const int32_t* perm, int k, int kp, int32_t* ids, float* dists,
                               cudaStream_t st)
{
    const int m = P.max_leaf;
    if (m <= 32) return launch_leaf_f32<1, kDT>(x, P, dp, T, perm, k, kp, ids, dists, st);
    if (m <= 64) return launch_leaf_f32<2, kDT>(x, P, dp, T, perm, k, kp, ids, dists, st);
    if (m <= 128) return launch_leaf_f32<4, kDT>(x, P, dp, T, perm, k, kp, ids, dists, st);
    if (m <= 256) return launch_leaf_f32<8, kDT>(x, P, dp, T, perm, k, kp, ids, dists, st);
    return launch_leaf_f32<16, kDT>(x, P, dp, T, perm, k, kp, ids, dists, st);
}

cudaError_t run_leaf_knn_f32(const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                             const int32_t* perm, int k, int kp, int32_t* ids, float* dists,
                             cudaStream_t st)
{
    if (kp > kCandCap) kp = kCandCap;
    if (x.dtype == kDtF16) return dispatch_ct<kDtF16>(x, P, dp, T, perm, k, kp, ids, dists, st);
    if (x.dtype == kDtU8) return dispatch_ct<kDtU8>(x, P, dp, T, perm, k, kp, ids, dists, st);
    return dispatch_ct<kDtF32>(x, P, dp, T, perm, k, kp, ids, dists, st);
}

}  // namespace knng
