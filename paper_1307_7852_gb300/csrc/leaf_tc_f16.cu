// Tensor-core leaf kernels instantiated for F16 point rows.
#include "leaf_tc_kernels.cuh"

namespace knng {
template cudaError_t leaf_tc_run<kDtF16>(int, const CUtensorMap&, const XDesc&, const TreePlan&, const DevPlan&, int,
                                        const int32_t*, int, void*, float*, float*, uint8_t*, int, int,
                                        const TcGeom&, int32_t*, float*, int*, int*, uint16_t*, uint8_t*,
                                        cudaStream_t);
}  // namespace knng
