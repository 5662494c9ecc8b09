// Output distribution of a batched build: the graphs of a group of point sets
// are computed over their concatenation (global point ids); every row goes
// back to its own set with the set's offset removed.
#include "knng_common.cuh"
#include "knng_internal.h"

namespace knng {

__global__ void scatter_batch_kernel(int64_t ng, int k, const BatchSet* __restrict__ sets, int nsets,
                                     const int32_t* __restrict__ gi, const float* __restrict__ gd)
{
    const int64_t total = ng * k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = e / k;
        const int slot = (int)(e - g * k);
        int lo = 0, hi = nsets - 1;  // last set with off <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (sets[mid].off <= g) lo = mid; else hi = mid - 1;
        }
        const BatchSet b = sets[lo];
        const int64_t i = g - b.off;
        const int32_t id = gi[e];
        b.ids[i * k + slot] = id >= 0 ? (int32_t)(id - b.off) : -1;
        b.dists[i * k + slot] = gd[e];
    }
}

cudaError_t run_scatter_batch(int64_t ng, int k, const BatchSet* sets, int nsets, const int32_t* gi,
                              const float* gd, cudaStream_t st)
{
    const int64_t work = ng * k;
    int blocks = (int)std::min<int64_t>((work + 255) / 256, (int64_t)num_sms() * 16);
    if (blocks < 1) blocks = 1;
    scatter_batch_kernel<<<blocks, 256, 0, st>>>(ng, k, sets, nsets, gi, gd);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace knng
