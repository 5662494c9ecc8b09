// Propagation rounds without any device allocation.
//
// Some callers cannot allocate device memory on their call path: a plugin
// inside an application whose memory manager already owns the device memory
// (where a cudaMalloc would fail or fight that manager), or a latency-critical
// loop that cannot afford the implicit synchronisation of cudaMalloc/cudaFree.
// knng_propagate needs a workspace for the lists between rounds and gets it
// from a handle; this entry point instead keeps those lists in one fixed,
// file-scope device array that the library reserves when it is loaded.  The
// array is modest (16 MiB) and every GPU that loads the library holds it
// until the process exits.
#include <mutex>

#include "../../include/knng.h"
#include "knng_internal.h"

namespace knng {

namespace {
constexpr int64_t kNoAllocMaxEntries = int64_t(1) << 19;  // n * k
constexpr int64_t kNoAllocMaxPoints = int64_t(1) << 19;   // n
constexpr size_t kListBytes = sizeof(int32_t) * kNoAllocMaxEntries;
constexpr size_t kFlagBytes = sizeof(unsigned long long) * kNoAllocMaxPoints;
// two (ids, dists, flags) buffers for the lists between rounds
constexpr size_t kScratchBytes = 2 * (2 * kListBytes + kFlagBytes);

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device.  The name of a
// __device__ array in host code is only a host-side stand-in, so the address
// is looked up once per device with that device current and kept for the
// life of the process (a device reset would invalidate it; the header asks
// for a process restart after one).
static int scratch_address(int dev, char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return KNNG_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return KNNG_ERR_CUDA;
        }
        g_addr[dev] = p;
    }
    *out = static_cast<char*>(g_addr[dev]);
    return KNNG_OK;
}

}  // namespace knng

using namespace knng;

extern "C" int knng_propagate_noalloc(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, int32_t k,
                                      int32_t rounds, const int32_t* ids_in, const float* dists_in, int32_t* ids,
                                      float* dists, void* stream)
{
    if (!X || !ids_in || !dists_in || !ids || !dists) return KNNG_ERR_INVALID_ARG;
    if (dtype != KNNG_DTYPE_F32 && dtype != KNNG_DTYPE_F16 && dtype != KNNG_DTYPE_U8) return KNNG_ERR_INVALID_ARG;
    if (n < 2 || d < 1 || d > 4096 || ld < d || ld >= (int64_t)1 << 31 || k < 1 || k > kMaxK) return KNNG_ERR_INVALID_ARG;
    if (rounds < 1 || rounds > 16) return KNNG_ERR_INVALID_ARG;
    if (n > kNoAllocMaxPoints || n * (int64_t)k > kNoAllocMaxEntries) return KNNG_ERR_LIMIT;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return KNNG_ERR_CUDA;
    }
    char* base = nullptr;
    const int r = scratch_address(dev, &base);
    if (r != KNNG_OK) return r;

    XDesc x;
    const size_t es = dtype == KNNG_DTYPE_F16 ? 2 : dtype == KNNG_DTYPE_U8 ? 1 : 4;
    const size_t align = dtype == KNNG_DTYPE_F16 ? 8 : dtype == KNNG_DTYPE_U8 ? 4 : 16;
    x.X = X;
    x.dtype = dtype;
    x.n = n;
    x.d = d;
    x.ld = ld;
    x.vec = ((uintptr_t)X % align == 0) && ((size_t)ld * es % align == 0);

    int32_t* bi[2];
    float* bd[2];
    unsigned long long* bf[2];
    for (int b = 0; b < 2; ++b) {
        char* p = base + (size_t)b * (2 * kListBytes + kFlagBytes);
        bi[b] = reinterpret_cast<int32_t*>(p);
        bd[b] = reinterpret_cast<float*>(p + kListBytes);
        bf[b] = reinterpret_cast<unsigned long long*>(p + 2 * kListBytes);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t* si = ids_in;
    const float* sd = dists_in;
    const unsigned long long* sf = nullptr;  // the input lists count as all new
    for (int rd = 0; rd < rounds; ++rd) {
        const bool last = rd == rounds - 1;
        int32_t* oi = last ? ids : bi[rd & 1];
        float* od = last ? dists : bd[rd & 1];
        unsigned long long* of = last ? nullptr : bf[rd & 1];
        const cudaError_t e = run_propagate(x, k, nullptr, si, sd, sf, oi, od, of, st);
        if (e != cudaSuccess) return KNNG_ERR_CUDA;
        si = oi;
        sd = od;
        sf = of;
    }
    return KNNG_OK;
}
