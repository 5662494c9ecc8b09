// Leaf graphs on the 5th-generation tensor cores (Sec. 3.1 of arXiv:1307.7852),
// host side: tile geometry of the TMA pipeline, the tensor map of the
// leaf-ordered quantised copy, the autotuner's candidate tiles, and the
// dispatch to the per-element-type instantiations of the kernels
// (leaf_tc_kernels.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "knng_common.cuh"
#include "knng_internal.h"
#include "leaf_tc_kernels.cuh"

namespace knng {

extern template cudaError_t leaf_tc_run<kDtF32>(int, const CUtensorMap&, const XDesc&, const TreePlan&, const DevPlan&,
                                                int, const int32_t*, int, void*, float*, float*, uint8_t*, int, int,
                                                const TcGeom&, int32_t*, float*, int*, int*, uint16_t*, uint8_t*,
                                                cudaStream_t);
extern template cudaError_t leaf_tc_run<kDtF16>(int, const CUtensorMap&, const XDesc&, const TreePlan&, const DevPlan&,
                                                int, const int32_t*, int, void*, float*, float*, uint8_t*, int, int,
                                                const TcGeom&, int32_t*, float*, int*, int*, uint16_t*, uint8_t*,
                                                cudaStream_t);
extern template cudaError_t leaf_tc_run<kDtU8>(int, const CUtensorMap&, const XDesc&, const TreePlan&, const DevPlan&,
                                               int, const int32_t*, int, void*, float*, float*, uint8_t*, int, int,
                                               const TcGeom&, int32_t*, float*, int*, int*, uint16_t*, uint8_t*,
                                                cudaStream_t);

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

static TcGeom tc_geometry(const TreePlan& P, int d, int prec, const TcTile* tile)
{
    TcGeom G{};
    const int elem = prec == 1 ? 2 : 1;
    const int slice = 128 / elem;
    const int dq = (d + slice - 1) / slice * slice;
    G.nK = dq / slice;
    G.N_load = (P.max_leaf + 15) & ~15;
    G.R_load = (P.max_leaf + 127) & ~127;
    G.box_rows = 128;  // R_load is a multiple of 128
    G.nbox = G.R_load / G.box_rows;
    G.stage_bytes = G.R_load * 128;
    G.ldD = ((G.N_load + 31) & ~31) + 1;
    const int s_max = std::max(1, std::min(std::min(G.nK, 4), (200 * 1024) / G.stage_bytes));
    if (tile && tile->S >= 1 && tile->RG >= 32) {
        G.S = std::min(tile->S, s_max);
        G.RG = tile->RG;
    } else {
        // default: deepest pipeline that fits; rows per epilogue group: 128,
        // 64 or 32 (a divisor of the 128-row block) within 72 KB
        G.S = s_max;
        G.RG = 128;
        while (G.RG > 32 && G.RG * G.ldD * 4 > 72 * 1024) G.RG >>= 1;
    }
    // the pipeline region is reused after the MMAs: by the row-per-thread
    // selection (kFastSmem), by the distance block of the warp-per-row path
    // and, past both, by the warps' selection scratch
    G.wsc_off = (std::max(G.RG * G.ldD * 4, 72 * 1024) + 15) & ~15;
    G.pipe_bytes = std::max(std::max(G.S * G.stage_bytes, G.wsc_off + kTcWarps * kLeafWarpScratch), kFastSmem);
    G.pipe_bytes = (G.pipe_bytes + 1023) & ~1023;
    G.smem = 1024 + G.pipe_bytes + 3 * G.N_load * 4 + 16 + (2 * G.S + 1) * 8 + 16;
    return G;
}

TcKey tc_key(const TreePlan& P, int d, int prec)
{
    const int elem = prec == 1 ? 2 : 1;
    const int slice = 128 / elem;
    return TcKey{prec, (d + slice - 1) / slice * 128, (P.max_leaf + 15) & ~15};
}

std::vector<TcTile> tc_candidates(const TreePlan& P, int d, int prec)
{
    std::vector<TcTile> out;
    const TcGeom base = tc_geometry(P, d, prec, nullptr);
    const int s_max = std::max(1, std::min(std::min(base.nK, 4), (200 * 1024) / base.stage_bytes));
    for (int S = 1; S <= s_max; ++S)
        for (int RG = 32; RG <= 128; RG <<= 1) {
            TcTile t{S, RG};
            if (tc_geometry(P, d, prec, &t).smem <= 220 * 1024) out.push_back(t);
        }
    return out;
}

cudaError_t run_leaf_knn_tc(const XDesc& x, const TreePlan& P, const DevPlan& dp, int T, const int32_t* perm,
                            int k, int kp, int prec, int32_t* ids, float* dists, int* err, Arena& ar,
                            cudaStream_t st, const TcTile* tile, int* all_exact, long long wait_cycles)
{
    const int elem = prec == 1 ? 2 : 1;
    const int slice = 128 / elem;
    const int dq = (x.d + slice - 1) / slice * slice;
    // rows of at least 1 KB in leaves of more than 256 points: one quantised
    // copy in point order that the leaf kernel gathers from (the per-tree
    // leaf-ordered copies would move T times the bytes through HBM); else a
    // leaf-ordered copy per tree, streamed by the tensor map
    const bool by_point = (int64_t)dq * elem >= 1024 && P.max_leaf > 256;
    const int64_t rows = by_point ? x.n : (int64_t)T * x.n;
    uint8_t* Xq = ar.take<uint8_t>((size_t)rows * dq * elem);
    float* qn = ar.take<float>((size_t)rows);
    float* qs = ar.take<float>((size_t)rows);
    uint8_t* qx = ar.take<uint8_t>((size_t)rows);
    if (kp > kTcCand) kp = kTcCand;
    // rows of leaves that are not exact are rescored by the staged kernel
    // (their candidates in [rows][kp] local indices, a flag per leaf)
    const bool staged = leaf_rescore_staged_ok(x, kp, P.max_leaf);
    const int nleaves = (int)P.leaf_off.size() - 1;
    uint16_t* cand = staged ? ar.take<uint16_t>((size_t)T * x.n * kp) : nullptr;
    uint8_t* leaf_flag = staged ? ar.take<uint8_t>((size_t)T * nleaves) : nullptr;
    if (!ar.base) return cudaSuccess;
    TcGeom G = tc_geometry(P, x.d, prec, tile);
    G.wait = wait_cycles > 0 ? wait_cycles : kWaitCycles;
    if (by_point) {
        G.xg = Xq;
        G.xg_ld = (int64_t)dq * elem;
    }
    if (G.smem > 227 * 1024) return cudaErrorInvalidConfiguration;

    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)dq, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)dq * elem};
    const cuuint32_t box[2] = {(cuuint32_t)slice, (cuuint32_t)G.box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult cr = enc(&map, prec == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, Xq, gdim,
                      gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;

    cudaError_t e;
    if (x.dtype == kDtF16)
        e = leaf_tc_run<kDtF16>(prec, map, x, P, dp, T, perm, dq, Xq, qn, qs, qx, k, kp, G, ids, dists, err, all_exact,
                                cand, leaf_flag, st);
    else if (x.dtype == kDtU8)
        e = leaf_tc_run<kDtU8>(prec, map, x, P, dp, T, perm, dq, Xq, qn, qs, qx, k, kp, G, ids, dists, err, all_exact,
                               cand, leaf_flag, st);
    else
        e = leaf_tc_run<kDtF32>(prec, map, x, P, dp, T, perm, dq, Xq, qn, qs, qx, k, kp, G, ids, dists, err, all_exact,
                                cand, leaf_flag, st);
    if (e == cudaSuccess && staged)
        e = run_leaf_rescore_staged(x, P, dp, T, perm, leaf_flag, cand, kp, k, ids, dists, st);
    return e;
}

}  // namespace knng
