// Exact byte copy of float point rows.  Descriptor sets such as SIFT hold
// integers 0..255 in float storage; such rows are stored again as bytes, and
// the kernels that gather rows at random (projection, propagation) read the
// copy: the same values in a quarter of the bytes.  One pass over X checks
// every entry; any entry that is not an integer in [0, 255] (NaN included)
// sets *bad and the copy is left unused.
#include "knng_common.cuh"
#include "knng_internal.h"

namespace knng {

__device__ __forceinline__ bool is_byte(float v)
{
    return v >= 0.f && v <= 255.f && v == rintf(v);
}
// the value of a byte entry (saturating and NaN-safe for the others, whose
// copy is never read)
__device__ __forceinline__ uint8_t to_byte(float v)
{
    return (uint8_t)min(__float2uint_rz(v), 255u);
}

// One thread per 4 bytes of a copied row (d4 = ldb / 4 groups per row; the
// padding bytes d .. ldb - 1 are written as zeros, so that 16-byte loads of a
// row see zeros past d).
__global__ void __launch_bounds__(256) byte_copy_kernel(RowLoader<kDtF32> L, int64_t n, int d4,
                                                        uint8_t* __restrict__ Xb, int64_t ldb, int* bad)
{
    const int64_t total = n * d4;
    bool ok = true;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = g / d4;
        const int j = 4 * (int)(g - i * d4);
        if (j >= L.d) {
            *reinterpret_cast<uchar4*>(Xb + i * ldb + j) = make_uchar4(0, 0, 0, 0);
            continue;
        }
        const float4 v = L.load4(i, j);  // zero past d
        ok = ok && is_byte(v.x) && is_byte(v.y) && is_byte(v.z) && is_byte(v.w);
        uint8_t* o = Xb + i * ldb + j;
        if (j + 3 < L.d) {
            *reinterpret_cast<uchar4*>(o) = make_uchar4(to_byte(v.x), to_byte(v.y), to_byte(v.z), to_byte(v.w));
        } else {
            *reinterpret_cast<uchar4*>(o) = make_uchar4(to_byte(v.x), j + 1 < L.d ? to_byte(v.y) : 0,
                                                        j + 2 < L.d ? to_byte(v.z) : 0, 0);
        }
    }
    if (__syncthreads_or(!ok) && threadIdx.x == 0) *bad = 1;
}

cudaError_t run_byte_copy(const XDesc& x, uint8_t* Xb, int64_t ldb, int* bad, cudaStream_t st)
{
    const int d4 = (int)(ldb / 4);
    const int64_t total = x.n * d4;
    const int64_t cap = (int64_t)num_sms() * 8;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, cap);
    RowLoader<kDtF32> L{x.X, x.ld, x.d, x.vec};
    byte_copy_kernel<<<grid, 256, 0, st>>>(L, x.n, d4, Xb, ldb, bad);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace knng
