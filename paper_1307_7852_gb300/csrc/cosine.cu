// Cosine metric (App. of arXiv:1307.7852, after the proof of Lemma 1: for the
// cosine distance a random projection builds the partition tree).  The rows
// are scaled to unit length in FP32 -- squared norm in the canonical order
// of the projection (lane partials over j = 128c + 4l + e, then the pairwise
// rounds 16..1), IEEE square root, one IEEE division per entry; a zero row
// stays zero -- and the method runs on the unit rows.  Between unit rows
// |u - v|^2 = 2 (1 - cos), so the squared distances are halved at the end to
// report 1 - cos.
#include "knng_common.cuh"
#include "knng_internal.h"

#include <type_traits>

namespace knng {

// One warp per row; out rows of ldo floats (ldo >= d, entries past d = 0).
template <int kDT>
__global__ void __launch_bounds__(256) normalize_rows_kernel(RowLoader<kDT> L, int64_t n, float* __restrict__ out,
                                                             int64_t ldo)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < n; i += nw) {
        float s = 0.f;
        for (int j = 4 * lane; j < L.d; j += 128) {
            const float4 v = L.load4(i, j);  // zero past d: fmaf(0, 0, s) = s
            s = fmaf(v.x, v.x, s);
            s = fmaf(v.y, v.y, s);
            s = fmaf(v.z, v.z, s);
            s = fmaf(v.w, v.w, s);
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(KNNG_FULL_MASK, s, o);
        const float r = sqrtf(s);
        float* u = out + i * ldo;
        for (int j = lane; j < ldo; j += 32) u[j] = (j < L.d && s > 0.f) ? L.load1(i, j) / r : 0.f;
    }
}

__global__ void scale_kernel(float* __restrict__ v, int64_t cnt, float f)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        v[i] *= f;
}

cudaError_t run_normalize_rows(const XDesc& x, float* out, int64_t ldo, cudaStream_t st)
{
    const int grid = (int)std::min<int64_t>((x.n + 7) / 8, (int64_t)num_sms() * 16);
    auto launch = [&](auto dt) {
        constexpr int kDT = decltype(dt)::value;
        RowLoader<kDT> L{x.X, x.ld, x.d, x.vec};
        normalize_rows_kernel<kDT><<<grid, 256, 0, st>>>(L, x.n, out, ldo);
    };
    if (x.dtype == kDtF16) launch(std::integral_constant<int, kDtF16>{});
    else if (x.dtype == kDtU8) launch(std::integral_constant<int, kDtU8>{});
    else launch(std::integral_constant<int, kDtF32>{});
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t run_scale(float* v, int64_t cnt, float f, cudaStream_t st)
{
    const int grid = (int)std::min<int64_t>((cnt + 255) / 256, (int64_t)num_sms() * 8);
    if (grid > 0) {
        scale_kernel<<<grid, 256, 0, st>>>(v, cnt, f);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace knng
