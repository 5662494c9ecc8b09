// Best-first neighbourhood propagation with a visit budget (Sec. 3.2 of
// arXiv:1307.7852), one synchronous pass over a frozen snapshot of the
// lists.  For every point p (one warp per point):
//  * p's own neighbours are visited first, in list order, and enter the
//    priority queue with their distance to p;
//  * the nearest unexpanded visited point is popped and its neighbours that
//    were not visited yet are visited, in its list order; and so on,
//  * until the queue is empty or `budget` points were visited (the budget
//    may end a list part way);
//  * p's new list is the k best visited points by (dist, id).
// Shared memory per warp: a hash set of visited ids (with p), the visited
// ids and their packed (dist, id) keys in visit order -- the queue is that
// array with a popped bit per entry, and a pop is a warp arg-min over it --
// and the selection scratch.  Distances are the canonical FP32 ones (float
// rows with an exact byte copy are scored on the copy).
#include "knng_common.cuh"
#include "knng_internal.h"

#include <type_traits>

namespace knng {

namespace {
struct BfLayout {
    int H, hshift, Bc;
    size_t per_warp;
};

BfLayout bf_layout(int budget)
{
    BfLayout L;
    L.Bc = (budget + 31) & ~31;
    int H = 64;
    while (H < 2 * (budget + 34)) H <<= 1;
    L.H = H;
    int lg = 0;
    while ((1 << lg) < H) ++lg;
    L.hshift = 32 - lg;
    // tab[H] | vid[Bc] | popped[Bc/32] | (8-aligned) vkey[Bc] | ws
    size_t b = sizeof(int) * (size_t)H + sizeof(int) * (size_t)L.Bc + sizeof(uint32_t) * (size_t)(L.Bc / 32);
    b = (b + 15) & ~(size_t)15;
    b += sizeof(uint64_t) * (size_t)L.Bc + kLeafWarpScratch;
    L.per_warp = (b + 15) & ~(size_t)15;
    return L;
}
}  // namespace

template <int kDT>
__global__ void __launch_bounds__(256, 2) propagate_bf_kernel(RowLoader<kDT> L, RowLoader<kDtU8> Lb,
                                                              const int* __restrict__ xb_bad, int64_t n, int k,
                                                              int budget, const int32_t* __restrict__ order,
                                                              const int32_t* __restrict__ ids_in,
                                                              int32_t* __restrict__ ids_out, float* __restrict__ d_out,
                                                              int H, int hshift, int Bc, int per_warp_bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char* base = smem_raw + (size_t)w * per_warp_bytes;
    int* tab = reinterpret_cast<int*>(base);
    int* vid = tab + H;
    uint32_t* popped = reinterpret_cast<uint32_t*>(vid + Bc);
    uint64_t* vkey = reinterpret_cast<uint64_t*>(((uintptr_t)(popped + Bc / 32) + 15) & ~(uintptr_t)15);
    unsigned char* ws = reinterpret_cast<unsigned char*>(vkey + Bc);
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws);
    uint64_t* keys = reinterpret_cast<uint64_t*>(ws + 1024);
    const uint32_t hmask = (uint32_t)H - 1;
    bool bytes = false;
    if constexpr (kDT == kDtF32) bytes = xb_bad && *xb_bad == 0;

    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t wi = gw; wi < n; wi += nw) {
        const int32_t p = order ? order[wi] : (int32_t)wi;
        for (int s = lane * 4; s < H; s += 128) *reinterpret_cast<int4*>(tab + s) = make_int4(-1, -1, -1, -1);
        for (int s = lane; s < Bc / 32; s += 32) popped[s] = 0u;
        __syncwarp();
        if (lane == 0) hash_insert(tab, (uint32_t)hshift, hmask, p);
        __syncwarp();
        int cnt = 0;
        // visits the lanes' ids o (-1: none) in lane order while the budget
        // lasts, and scores them (collective)
        auto visit = [&](int32_t o) {
            const bool fresh = o >= 0 && hash_insert(tab, (uint32_t)hshift, hmask, o);
            const uint32_t b = __ballot_sync(KNNG_FULL_MASK, fresh);
            const int pos = cnt + __popc(b & lanemask_lt());
            if (fresh && pos < budget) vid[pos] = o;
            const int end = min(cnt + __popc(b), budget);
            __syncwarp();
            for (int c0 = cnt; c0 < end; c0 += 32) {
                const int nb = min(32, end - c0);
                float dd;
                if (kDT == kDtF32 && bytes) dd = warp_canon_dist32(Lb, p, vid + c0, nb);
                else dd = warp_canon_dist32(L, p, vid + c0, nb);
                if (lane < nb) vkey[c0 + lane] = pack_key(dd, (uint32_t)vid[c0 + lane]);
            }
            cnt = end;
            __syncwarp();
        };
        for (int e0 = 0; e0 < k; e0 += 32) {
            const int e = e0 + lane;
            int32_t o = e < k ? ids_in[(int64_t)p * k + e] : -1;
            if (o >= n) o = -1;  // ids outside [0, n) are empty slots
            visit(o);
        }
        while (cnt < budget) {
            // pop the nearest visited point not expanded yet
            uint64_t best = kKeyMax;
            int bi = -1;
            for (int i = lane; i < cnt; i += 32) {
                if (((popped[i >> 5] >> (i & 31)) & 1u) == 0u && vkey[i] < best) {
                    best = vkey[i];
                    bi = i;
                }
            }
            uint64_t wbest = best;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const uint64_t other = __shfl_xor_sync(KNNG_FULL_MASK, wbest, o);
                wbest = other < wbest ? other : wbest;
            }
            if (wbest == kKeyMax) break;  // queue empty
            const int owner = __ffs(__ballot_sync(KNNG_FULL_MASK, best == wbest)) - 1;
            const int idx = __shfl_sync(KNNG_FULL_MASK, bi, owner);
            __syncwarp();
            if (lane == 0) popped[idx >> 5] |= 1u << (idx & 31);
            const int32_t u = vid[idx];
            __syncwarp();
            for (int f0 = 0; f0 < k && cnt < budget; f0 += 32) {
                const int f = f0 + lane;
                int32_t o = f < k ? ids_in[(int64_t)u * k + f] : -1;
                if (o >= n) o = -1;
                visit(o);
            }
        }
        auto key = [&](int i) -> uint64_t { return vkey[i]; };
        const int nsel = warp_topk_sorted<16>(key, cnt, k, keys, keys + 64, hist);
        __syncwarp();
        for (int i = lane; i < k; i += 32) {
            const bool ok = i < nsel;
            ids_out[(int64_t)p * k + i] = ok ? (int32_t)(uint32_t)keys[i] : -1;
            d_out[(int64_t)p * k + i] = ok ? unord_key((uint32_t)(keys[i] >> 32)) : __int_as_float(0x7f800000);
        }
        __syncwarp();
    }
}

cudaError_t run_propagate_best_first(const XDesc& x, int k, int budget, const int32_t* order, const int32_t* ids_in,
                                     int32_t* ids, float* dists, cudaStream_t st)
{
    if (budget < k || budget > 512 || k > 64) return cudaErrorInvalidValue;
    const BfLayout BL = bf_layout(budget);
    int warps = (int)((200 * 1024) / BL.per_warp);
    if (warps > 8) warps = 8;
    if (warps < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = BL.per_warp * warps;
    cudaError_t e = cudaSuccess;
    auto launch = [&](auto dt) {
        constexpr int kDT = decltype(dt)::value;
        auto kern = propagate_bf_kernel<kDT>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t blocks = (int64_t)num_sms() * per_sm;
        const int64_t need = (x.n + warps - 1) / warps;
        if (blocks > need) blocks = need;
        RowLoader<kDT> rl{x.X, x.ld, x.d, x.vec};
        const RowLoader<kDtU8> rb{x.Xb, x.ldb, x.d, true};
        kern<<<(int)blocks, warps * 32, smem, st>>>(rl, rb, x.xb_bad, x.n, k, budget, order, ids_in, ids, dists,
                                                    BL.H, BL.hshift, BL.Bc, (int)BL.per_warp);
        note_launches(1);
        e = cudaGetLastError();
    };
    if (x.dtype == kDtF16) launch(std::integral_constant<int, kDtF16>{});
    else if (x.dtype == kDtU8) launch(std::integral_constant<int, kDtU8>{});
    else launch(std::integral_constant<int, kDtF32>{});
    return e;
}

}  // namespace knng
