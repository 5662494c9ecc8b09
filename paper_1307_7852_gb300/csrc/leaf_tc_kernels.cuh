#pragma once
// Leaf graphs on the 5th-generation tensor cores (Sec. 3.1 of arXiv:1307.7852:
// a brute-force k-NN graph inside every leaf), reduced-precision candidate
// stage with exact FP32 rescoring.
//
//  1. gather_quant: writes every tree's points in leaf order as bfloat16 (or
//     E4M3 codes with one FP32 scale per row), rows zero-padded to whole
//     128-byte K slices, with the squared norm of each quantised row.
//  2. leaf_tc: one CTA per (tree, leaf, block of 128 rows).  A single thread
//     streams the leaf's rows through a TMA pipeline (128-byte swizzled
//     tiles, mbarrier completion) and issues tcgen05.mma with the CTA's 128
//     rows as A and all leaf rows as B (A is a slice of the B tile), so the
//     Gram block S = X_rows X_leaf^T accumulates in TMEM in FP32.  The four
//     warps read their TMEM lanes back (tcgen05.ld), form
//     D~ = |x|^2 + |y|^2 - 2 S (with the row scales for E4M3) and, one warp
//     per row, select the k' best candidates, rescore them with the canonical
//     FP32 distance on the original rows and keep the k best.
// Kernels and per-element-type launchers; the host side (tile geometry,
// tensor map) is in leaf_tc.cu, one instantiation per element type in
// leaf_tc_f32.cu / leaf_tc_f16.cu / leaf_tc_u8.cu.
// Every mbarrier wait is bounded; a CTA that gives up records the failure in
// the error word, waits for its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "knng_common.cuh"
#include "knng_internal.h"
#include "tc_ptx.cuh"

namespace knng {

namespace {
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at GB300 clocks
constexpr int kTcThreads = 256;  // 8 warps: warps w and w+4 share TMEM lanes 32(w%4)..+31
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kTcCand = 128;
}  // namespace

// ---------------------------------------------------------------------------
// 1. leaf-order gather and quantisation
// ---------------------------------------------------------------------------
//     For bfloat16 every row also gets an exactness bit: set when all its
//     entries are integers of magnitude <= 256 and its squared norm is below
//     2^23.  Between two such rows every bfloat16 value, product and partial
//     sum of the Gram is an integer below 2^24, exact in FP32, so the
//     candidate distance |x|^2 + |y|^2 - 2 x.y equals the true squared
//     distance, which is also what the canonical FP32 distance returns.
template <int PREC, class Loader>
__device__ __forceinline__ void gather_quant_body(const Loader& L, int64_t rows, const int32_t* __restrict__ perm,
                                                  int dq, void* __restrict__ out, float* __restrict__ nrm,
                                                  float* __restrict__ scl, uint8_t* __restrict__ exact)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = gw; r < rows; r += nw) {
        const int32_t id = perm ? perm[r] : (int32_t)r;
        float s = 0.f;
        bool ex = true;
        if (PREC == 1) {
            __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out) + r * dq;
            for (int j = 4 * lane; j < dq; j += 128) {
                const float4 v = j < L.d ? L.load4(id, j) : make_float4(0.f, 0.f, 0.f, 0.f);
                ex &= v.x == rintf(v.x) && v.y == rintf(v.y) && v.z == rintf(v.z) && v.w == rintf(v.w);
                ex &= fabsf(v.x) <= 256.f && fabsf(v.y) <= 256.f && fabsf(v.z) <= 256.f && fabsf(v.w) <= 256.f;
                __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
                __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
                const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
                s = fmaf(fa.x, fa.x, s); s = fmaf(fa.y, fa.y, s);
                s = fmaf(fb.x, fb.x, s); s = fmaf(fb.y, fb.y, s);
                uint2 u;
                u.x = *reinterpret_cast<uint32_t*>(&a);
                u.y = *reinterpret_cast<uint32_t*>(&b);
                *reinterpret_cast<uint2*>(o + j) = u;
            }
        } else {
            float mx = 0.f;
            for (int j = 4 * lane; j < L.d; j += 128) {
                const float4 v = L.load4(id, j);
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(KNNG_FULL_MASK, mx, o));
            const float sc = mx > 0.f ? mx / 448.0f : 1.0f;
            uint8_t* o = static_cast<uint8_t*>(out) + r * dq;
            for (int j = 4 * lane; j < dq; j += 128) {
                const float4 v = j < L.d ? L.load4(id, j) : make_float4(0.f, 0.f, 0.f, 0.f);
                const __nv_fp8_e4m3 q0(v.x / sc), q1(v.y / sc), q2(v.z / sc), q3(v.w / sc);
                const float f0 = float(q0), f1 = float(q1), f2 = float(q2), f3 = float(q3);
                s = fmaf(f0, f0, s); s = fmaf(f1, f1, s); s = fmaf(f2, f2, s); s = fmaf(f3, f3, s);
                const uint32_t u = (uint32_t)q0.__x | ((uint32_t)q1.__x << 8) | ((uint32_t)q2.__x << 16) |
                                   ((uint32_t)q3.__x << 24);
                *reinterpret_cast<uint32_t*>(o + j) = u;
            }
            if (lane == 0) scl[r] = sc;
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(KNNG_FULL_MASK, s, o);
        ex = __all_sync(KNNG_FULL_MASK, ex);
        if (lane == 0) {
            nrm[r] = s;
            exact[r] = (PREC == 1 && ex && s < 8388608.0f) ? 1 : 0;
        }
    }
}

// Byte rows to bfloat16 (16-byte aligned rows padded with zeros to
// multiples of 16 bytes, d <= 256): a group of LPR lanes per row, 16 bytes a
// lane, two rows in flight per group.  A byte b becomes the float 2^23 + b
// by a byte permute, 2^23 comes off with a packed subtract, and the pair
// rounds to bfloat16 exactly (b < 2^8).  The squared norm is the exact
// integer sum of b^2 (dp4a), below 2^24, so it equals the FP32 sum of any
// order; every row of bytes is exact when that norm is below 2^23.
template <int LPR>
__device__ __forceinline__ void gather_bytes_bf16(const RowLoader<kDtU8>& Lb, int64_t rows,
                                                  const int32_t* __restrict__ perm, int dq,
                                                  __nv_bfloat16* __restrict__ out, float* __restrict__ nrm,
                                                  uint8_t* __restrict__ exact)
{
    const int lane = threadIdx.x & 31, q = lane % LPR;
    const unsigned gmask = LPR == 32 ? 0xFFFFFFFFu : (((1u << LPR) - 1u) << (lane - q));
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / LPR;
    const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LPR;
    const int d16 = (Lb.d + 15) & ~15;
    const bool has = 16 * q < d16, put = 16 * q < dq;
    const uint8_t* X = static_cast<const uint8_t*>(Lb.X);
    const float2 off = make_float2(-8388608.0f, -8388608.0f);
    auto cvt = [&](uint32_t w, uint32_t& lo, uint32_t& hi) {
        const float2 a = __fadd2_rn(make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u)),
                                                __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7541u))),
                                    off);
        const float2 b = __fadd2_rn(make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7542u)),
                                                __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7543u))),
                                    off);
        const __nv_bfloat162 ha = __floats2bfloat162_rn(a.x, a.y), hb = __floats2bfloat162_rn(b.x, b.y);
        lo = *reinterpret_cast<const uint32_t*>(&ha);
        hi = *reinterpret_cast<const uint32_t*>(&hb);
    };
    for (int64_t r0 = grp; r0 < rows; r0 += 2 * ngrp) {
        const int64_t r1 = r0 + ngrp;
        const bool two = r1 < rows;
        const int32_t id0 = perm ? perm[r0] : (int32_t)r0;
        const int32_t id1 = two ? (perm ? perm[r1] : (int32_t)r1) : id0;
        uint4 u[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
        if (has) {
            u[0] = __ldg(reinterpret_cast<const uint4*>(X + Lb.row_off(id0) + 16 * q));
            u[1] = __ldg(reinterpret_cast<const uint4*>(X + Lb.row_off(id1) + 16 * q));
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int64_t r = e ? r1 : r0;
            uint32_t acc = 0u;
            acc = __dp4a(u[e].x, u[e].x, acc);
            acc = __dp4a(u[e].y, u[e].y, acc);
            acc = __dp4a(u[e].z, u[e].z, acc);
            acc = __dp4a(u[e].w, u[e].w, acc);
            uint4 o0, o1;
            cvt(u[e].x, o0.x, o0.y);
            cvt(u[e].y, o0.z, o0.w);
            cvt(u[e].z, o1.x, o1.y);
            cvt(u[e].w, o1.z, o1.w);
#pragma unroll
            for (int sh = LPR / 2; sh >= 1; sh >>= 1) acc += __shfl_xor_sync(gmask, acc, sh, LPR);
            if (e == 0 || two) {
                if (put) {
                    uint4* dst = reinterpret_cast<uint4*>(out + r * dq + 16 * q);
                    dst[0] = o0;
                    dst[1] = o1;
                }
                if (q == 0) {
                    nrm[r] = (float)acc;
                    exact[r] = acc < 8388608u ? 1 : 0;
                }
            }
        }
    }
}

// Float rows whose byte copy is exact (*xb_bad == 0) are read from the copy;
// for bfloat16, rows of bytes (the copy, or aligned byte input) of at most
// 256 entries take the byte conversion above.
template <int PREC, int kDT>
__global__ void __launch_bounds__(256) gather_quant_kernel(RowLoader<kDT> L, RowLoader<kDtU8> Lb,
                                                           const int* __restrict__ xb_bad, int64_t rows,
                                                           const int32_t* __restrict__ perm, int dq,
                                                           void* __restrict__ out, float* __restrict__ nrm,
                                                           float* __restrict__ scl, uint8_t* __restrict__ exact,
                                                           bool u8_aligned)
{
    auto bytes_bf16 = [&](const RowLoader<kDtU8>& B) {
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(out);
        if (dq <= 64) gather_bytes_bf16<4>(B, rows, perm, dq, o, nrm, exact);
        else if (dq <= 128) gather_bytes_bf16<8>(B, rows, perm, dq, o, nrm, exact);
        else gather_bytes_bf16<16>(B, rows, perm, dq, o, nrm, exact);
    };
    if constexpr (kDT == kDtF32) {
        if (xb_bad && *xb_bad == 0) {
            if (PREC == 1 && Lb.d <= 256) bytes_bf16(Lb);
            else gather_quant_body<PREC>(Lb, rows, perm, dq, out, nrm, scl, exact);
            return;
        }
    }
    if constexpr (kDT == kDtU8) {
        if (PREC == 1 && u8_aligned && L.d <= 256) {
            bytes_bf16(L);
            return;
        }
    }
    gather_quant_body<PREC>(L, rows, perm, dq, out, nrm, scl, exact);
}

// ---------------------------------------------------------------------------
// 2. Gram on tcgen05 + selection + rescoring
// ---------------------------------------------------------------------------
struct TcGeom {
    int N_load;      // largest MMA N over the leaves (multiple of 16)
    int R_load;      // rows loaded per K slice (multiple of 128)
    int box_rows;    // rows per TMA box (<= 256)
    int nbox;        // boxes per K slice
    int nK;          // K slices of 128 bytes
    int S;           // pipeline stages
    int stage_bytes;
    int RG;          // epilogue rows per group
    int ldD;         // row stride of the distance block (floats)
    int pipe_bytes;
    int wsc_off;     // offset of the warps' selection scratch in the pipeline region
    int smem;
    long long wait;  // limit of the producer's waits (copies landed, stage released)
    const uint8_t* xg = nullptr;  // quantised rows in point order (else the leaf-ordered copy)
    int64_t xg_ld = 0;            // their stride in bytes
};

// Bitonic sorting network on a thread's own registers (N a power of two;
// every index is a compile-time constant after unrolling).
template <class T, int N>
__device__ __forceinline__ void reg_bitonic_sort(T (&v)[N])
{
#pragma unroll
    for (int kk = 2; kk <= N; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & kk) == 0;
                    const T a = v[i], b = v[l];
                    const bool sw = up ? (b < a) : (a < b);
                    v[i] = sw ? b : a;
                    v[l] = sw ? a : b;
                }
            }
        }
    }
}

// Shared memory of the row-per-thread selection (reusing the pipeline):
// sorted group minima [32][256] u32 (later the halves' sorted runs
// [2][16][128] u64) and candidate lists [32][256] u64 (later the rows'
// merged lists [32][128] u64).
constexpr int kFastSmem = 32 * kTcThreads * 4 + 32 * kTcThreads * 8;

template <int PREC, int PER, int kDT>
__global__ void __launch_bounds__(kTcThreads, PER == 16 ? 1 : 2) leaf_tc_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                RowLoader<kDT> L, int64_t n,
                                                                const int32_t* __restrict__ perm,
                                                                const int32_t* __restrict__ leaf_off,
                                                                int nleaves, const float* __restrict__ qnrm,
                                                                const float* __restrict__ qscl,
                                                                const uint8_t* __restrict__ qexact, int k, int kp,
                                                                TcGeom G, int32_t* __restrict__ out_ids,
                                                                float* __restrict__ out_d, int* err, int* all_exact,
                                                                uint16_t* __restrict__ cand_out,
                                                                uint8_t* __restrict__ leaf_flag)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // the quantised rows in point order (null: the leaf-ordered copy of the
    // tensor map; leaves of more than 256 points only)
    const uint8_t* __restrict__ xg = PER == 16 ? G.xg : nullptr;
    const int64_t xg_ld = G.xg_ld;
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* pipe = base;
    float* Dblk = reinterpret_cast<float*>(pipe);
    int32_t* lid = reinterpret_cast<int32_t*>(base + G.pipe_bytes);
    float* qn = reinterpret_cast<float*>(lid + G.N_load);
    float* qs = qn + G.N_load;
    unsigned char* wsc = pipe + G.wsc_off;  // used only after the MMAs
    uint64_t* bars = reinterpret_cast<uint64_t*>(((uintptr_t)(qs + G.N_load) + 15) & ~(uintptr_t)15);
    uint64_t* full = bars;
    uint64_t* empty = bars + G.S;
    uint64_t* done = bars + 2 * G.S;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int abort_flag;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int t = blockIdx.y;
    const int RB = gridDim.x / nleaves;
    const int leaf = blockIdx.x / RB;
    const int r0 = (blockIdx.x % RB) * 128;
    const int off = leaf_off[leaf];
    const int m = leaf_off[leaf + 1] - off;
    if (r0 >= m) return;
    const int Nm = min(G.N_load, (m + 15) & ~15);
    const int N0 = min(Nm, 256), N1 = Nm - N0;
    uint32_t ncols = 32;
    while ((int)ncols < Nm) ncols <<= 1;

    if (tid == 0) {
        for (int s = 0; s < G.S; ++s) {
            // copies by the tensor map: one arrival (with the bytes); copies
            // of the rows by the threads: every thread arrives
            tc::mbar_init(&full[s], xg ? kTcThreads : 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_mbar_init();
        abort_flag = 0;
        if (!xg) tc::prefetch_tmap(&tmap);
    }
    if (w == 0) {
        tc::tmem_alloc(tslot, ncols);
        tc::tmem_relinquish();
    }
    const int64_t rowbase = (int64_t)t * n + off;
    bool ex = PREC == 1;
    for (int j = tid; j < G.N_load; j += kTcThreads) {
        const bool v = j < m;
        const int32_t id = v ? perm[rowbase + j] : 0;
        lid[j] = id;
        // norms, scales and exactness by leaf position (leaf-ordered copy)
        // or by point (the copy in point order)
        const int64_t qi = xg ? (int64_t)id : rowbase + j;
        qn[j] = v ? qnrm[qi] : 0.f;
        qs[j] = (PREC == 2 && v) ? qscl[qi] : 1.f;
        if (v) ex = ex && qexact[qi];
    }
    tc::fence_before_sync();
    // the whole leaf is exact: candidate distances are final, no rescoring
    const bool exact_leaf = __syncthreads_and(ex) != 0;
    if (tid == 0 && all_exact && !exact_leaf) atomicAnd(all_exact, 0);
    // with cand_out, rows of a leaf that is not exact leave their candidates
    // (local indices) for the staged FP32 rescoring kernel instead
    const bool to_cands = cand_out != nullptr && !exact_leaf;
    if (leaf_flag && tid == 0 && r0 == 0) leaf_flag[(int64_t)t * nleaves + leaf] = exact_leaf ? 1 : 0;
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;

    // ---- producer + MMA issuer ----------------------------------------------
    constexpr uint32_t fmt = PREC == 1 ? 1u : 0u;  // BF16 | E4M3
    // the MMAs of K slice kc in stage s (one thread), then their commit to
    // the stage's "empty" barrier
    auto mma_slice = [&](int kc, int s) {
        const uint32_t id0 = tc::make_idesc(fmt, 128, (uint32_t)N0);
        const uint32_t id1 = tc::make_idesc(fmt, 128, (uint32_t)(N1 > 0 ? N1 : 16));
        const uint32_t sa = tc::smem_u32(pipe + (size_t)s * G.stage_bytes);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = tc::sw128_desc(sa + (uint32_t)r0 * 128u + (uint32_t)kk * 32u);
            const uint64_t bd0 = tc::sw128_desc(sa + (uint32_t)kk * 32u);
            const uint32_t acc = (kc | kk) ? 1u : 0u;
            if (PREC == 1) tc::mma_f16(tbase, ad, bd0, id0, acc);
            else tc::mma_f8(tbase, ad, bd0, id0, acc);
            if (N1 > 0) {
                const uint64_t bd1 = tc::sw128_desc(sa + 256u * 128u + (uint32_t)kk * 32u);
                if (PREC == 1) tc::mma_f16(tbase + 256, ad, bd1, id1, acc);
                else tc::mma_f8(tbase + 256, ad, bd1, id1, acc);
            }
        }
        tc::mma_commit(&empty[s]);
    };
    if (PER != 16 || !xg) {
        // the leaf's rows are contiguous in the leaf-ordered copy: one thread
        // streams the K slices by the tensor map and issues the MMAs
        if (tid == 0) {
            const int xstep = PREC == 1 ? 64 : 128;  // elements per 128-byte K slice
            const int64_t yrow = rowbase;
            int loaded = 0, consumed = 0;
            bool ok = true;
            auto load = [&](int kc) {
                const int s = kc % G.S;
                tc::mbar_arrive_expect_tx(&full[s], (uint32_t)(G.nbox * G.box_rows * 128));
                for (int b = 0; b < G.nbox; ++b)
                    tc::tma_load_2d(pipe + (size_t)s * G.stage_bytes + (size_t)b * G.box_rows * 128, &tmap,
                                    &full[s], kc * xstep, (int)(yrow + (int64_t)b * G.box_rows));
            };
            for (; loaded < min(G.S, G.nK); ++loaded) load(loaded);
            for (int kc = 0; kc < G.nK; ++kc) {
                const int s = kc % G.S;
                const uint32_t ph = (uint32_t)(kc / G.S) & 1u;
                if (!tc::mbar_wait(&full[s], ph, G.wait)) { ok = false; break; }
                consumed = kc + 1;
                tc::fence_after_sync();
                mma_slice(kc, s);
                if (kc + G.S < G.nK) {
                    if (!tc::mbar_wait(&empty[s], ph, G.wait)) { ok = false; break; }
                    load(kc + G.S);
                    ++loaded;
                }
            }
            tc::mma_commit(done);
            if (!ok) {
                abort_flag = 1;
                atomicExch(err, 1);
                // wait (bounded, under the long limit whatever G.wait is) for
                // the copies this CTA still has in flight
                for (int kc = consumed; kc < loaded; ++kc)
                    tc::mbar_wait(&full[kc % G.S], (uint32_t)(kc / G.S) & 1u, kWaitCycles);
            }
        }
    } else if constexpr (PER == 16) {
        // rows from the copy in point order (rows of xg_ld bytes; leaves of
        // more than 256 points, one CTA per SM): every
        // thread copies 16-byte chunks of the leaf's rows into the stage, in
        // the 128-byte swizzled layout (chunk c of row r at c ^ (r mod 8)),
        // S - 1 slices ahead; once a slice has landed each thread fences its
        // writes for the tensor core and arrives; one thread waits for all
        // and issues the slice's MMAs.  Rows past the leaf read zeros.
        // Thread tid copies chunk c = tid mod 8 of rows tid / 8 + 32 i: the
        // same rows in every slice, so their addresses are formed once, and
        // r mod 8 (the swizzle) is the same for all of them.
        bool ok = true;
        const int cq = tid & 7, rq = tid >> 3;
        const int nri = G.R_load / 32;  // rows per thread (R_load <= 512)
        const uint8_t* rp[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int r = rq + 32 * i;
            rp[i] = (i < nri && r < m) ? xg + (int64_t)lid[r] * xg_ld + 16 * cq : nullptr;
        }
        const size_t dst0 = (size_t)rq * 128 + ((cq ^ (rq & 7)) << 4);
        for (int kc = 0; kc < G.nK + G.S - 1; ++kc) {
            if (kc < G.nK) {
                const int s = kc % G.S;
                if (kc >= G.S && !tc::mbar_wait(&empty[s], (uint32_t)((kc / G.S) - 1) & 1u, G.wait)) ok = false;
                unsigned char* dst = pipe + (size_t)s * G.stage_bytes + dst0;
                if (ok) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (i < nri)
                            cp_async16(dst + (size_t)i * 4096, rp[i] ? rp[i] + (int64_t)kc * 128 : xg,
                                       rp[i] ? 16 : 0);
                }
                cp_async_commit();
            }
            const int kd = kc - (G.S - 1);
            if (kd >= 0) {
                const int pend = min(G.S - 1, G.nK - 1 - kd);  // later slices may stay in flight
                if (pend >= 3) cp_async_wait<3>();
                else if (pend == 2) cp_async_wait<2>();
                else if (pend == 1) cp_async_wait<1>();
                else cp_async_wait<0>();
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(&full[kd % G.S]);
                if (tid == 0) {
                    if (tc::mbar_wait(&full[kd % G.S], (uint32_t)(kd / G.S) & 1u, G.wait)) {
                        tc::fence_after_sync();
                        mma_slice(kd, kd % G.S);
                    } else {
                        ok = false;
                    }
                }
            }
        }
        if (tid == 0) tc::mma_commit(done);
        if (!ok) {
            abort_flag = 1;
            atomicExch(err, 1);
        }
    }
    __syncthreads();
    if (!tc::mbar_wait(done, 0, kWaitCycles)) {
        abort_flag = 1;
        atomicExch(err, 1);
    }
    tc::fence_after_sync();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // pipeline smem is reused below
    __syncthreads();

    // ---- epilogue -------------------------------------------------------
    // Row per thread first: thread (quad, half) owns row 32 quad + lane and
    // the column chunks 32 half + 64 i of it.  Pass 1 takes the minimum of
    // the distances over the columns with the same position in their chunk
    // (32 groups per thread), sorts them; the want-th smallest of the 64
    // minima of a row (both halves) bounds the row's answer.  Pass 2 lists
    // the columns up to that bound, and the half-0 thread sorts the union of
    // the row's two lists (at most 32) with a register network.  Rows whose
    // lists overflow, and all rows when more than 32 candidates are wanted,
    // take the warp-per-row path below.
    if (!abort_flag) {
        const int quad = w & 3, half = w >> 2;
        const int lr = 32 * quad + lane;
        const int iloc = r0 + lr;
        const bool row_ok = iloc < m;
        const int kw = exact_leaf ? k : kp;
        const int want = min(kw, m - 1);
        uint32_t* gsh = reinterpret_cast<uint32_t*>(pipe);                     // [32][256]
        uint64_t* cand = reinterpret_cast<uint64_t*>(pipe + 32 * kTcThreads * 4);  // [32][256]
        __shared__ int ccount[kTcThreads];
        __shared__ unsigned char rowflag[128];
        __shared__ int any_overflow;
        const bool fast = want <= 32;
        if (tid == 0) any_overflow = fast ? 0 : 1;
        if (tid < 128) rowflag[tid] = fast ? 0 : 1;
        __syncthreads();
        const int il = min(iloc, G.N_load - 1);
        const float ni = qn[il], si = qs[il];
        const uint32_t trow = tbase + ((uint32_t)(32 * quad) << 16);
        // the distances of one chunk of 32 columns (FP32, as the keys take
        // them); columns past the leaf (last chunk) and the row's own column
        // read +inf.  The own column is column `lane` of the chunk r0 + 32 quad,
        // the same chunk for the whole warp.
        const int cself = r0 + 32 * quad;
        const float kInf = __int_as_float(0x7f800000);
        auto chunk_dv = [&](const uint32_t (&r)[32], int c0, float (&dv)[32]) {
            if (PREC == 1) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float4 q = *reinterpret_cast<const float4*>(qn + c0 + 4 * i);
                    const float qv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2)
                        dv[4 * i + e2] = ni + qv[e2] - 2.f * __uint_as_float(r[4 * i + e2]);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    const int jj = min(c0 + e, G.N_load - 1);
                    dv[e] = si * si * ni + qs[jj] * qs[jj] * qn[jj] - 2.f * si * qs[jj] * __uint_as_float(r[e]);
                }
            }
            if (c0 + 32 > m) {
#pragma unroll
                for (int e = 0; e < 32; ++e) dv[e] = (c0 + e < m) ? dv[e] : kInf;
            }
            if (c0 == cself) {
#pragma unroll
                for (int e = 0; e < 32; ++e) dv[e] = (e == lane) ? kInf : dv[e];
            }
        };
        // the thread's chunks c0 = 32 half + 64 i in order; with leaves of
        // more than 256 points (one CTA per SM, registers to spare) the next
        // chunk's tensor-memory load is in flight while one is processed
        auto for_chunks = [&](auto&& body) {
            if constexpr (PER == 16) {
                uint32_t ra[32], rb[32];
                int c0 = 32 * half;
                if (c0 < Nm) {
                    tc::tmem_ld32(trow + (uint32_t)c0, ra);
                    tc::tmem_ld_wait(ra);
                }
                for (; c0 < Nm; c0 += 128) {
                    const int c1 = c0 + 64, c2 = c0 + 128;
                    if (c1 < Nm) tc::tmem_ld32(trow + (uint32_t)c1, rb);
                    body(ra, c0);
                    if (c1 >= Nm) break;
                    tc::tmem_ld_wait(rb);
                    if (c2 < Nm) tc::tmem_ld32(trow + (uint32_t)c2, ra);
                    body(rb, c1);
                    if (c2 < Nm) tc::tmem_ld_wait(ra);
                }
            } else {
                for (int c0 = 32 * half; c0 < Nm; c0 += 64) {
                    uint32_t r[32];
                    tc::tmem_ld32(trow + (uint32_t)c0, r);
                    tc::tmem_ld_wait();
                    body(r, c0);
                }
            }
        };
        if (fast) {
            // pass 1: group minima of the distances (a float bound: keys
            // order as their distances do, so the want-th smallest minimum
            // bounds the row's answer as its key would)
            float gm[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) gm[e] = kInf;
            for_chunks([&](const uint32_t (&r)[32], int c0) {
                float dv[32];
                chunk_dv(r, c0, dv);
#pragma unroll
                for (int e = 0; e < 32; ++e) gm[e] = fminf(gm[e], dv[e]);
            });
            reg_bitonic_sort(gm);
            float* gshf = reinterpret_cast<float*>(gsh);
#pragma unroll
            for (int e = 0; e < 32; ++e) gshf[e * kTcThreads + tid] = gm[e];
            __syncthreads();
            // the want-th smallest of the row's 64 minima (two sorted lists
            // A, B): binary search for the number i of them taken from A, the
            // smallest i with A[i] >= B[want - i - 1]
            const int ptid = tid ^ 128;
            float tau;
            {
                int lo = max(0, want - 32), hi = min(want, 32);
                while (lo < hi) {
                    const int i = (lo + hi) >> 1;
                    const float a = gshf[i * kTcThreads + tid];  // i < hi <= 32
                    const float b = gshf[(want - i - 1) * kTcThreads + ptid];
                    if (a >= b) hi = i;
                    else lo = i + 1;
                }
                const float ta = lo > 0 ? gshf[(lo - 1) * kTcThreads + tid] : -kInf;
                const float tb = want - lo > 0 ? gshf[(want - lo - 1) * kTcThreads + ptid] : -kInf;
                tau = fmaxf(ta, tb);
                if (tau == kInf) tau = __int_as_float(0x7f7fffff);  // the invalid columns stay out
            }
            // pass 2: the candidates up to the bound
            int c = 0;
            for_chunks([&](const uint32_t (&r)[32], int c0) {
                float dv[32];
                chunk_dv(r, c0, dv);
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    if (dv[e] <= tau) {
                        if (c < 32) cand[c * kTcThreads + tid] = ((uint64_t)ord_key(dv[e]) << 32) | (uint32_t)(c0 + e);
                        ++c;
                    }
                }
            });
            if (c > 32 && row_ok) {
                rowflag[lr] = 1;
                any_overflow = 1;
            }
            ccount[tid] = min(c, 32);
            __syncthreads();
            // the union of the row's two lists (slots: list A, then list B),
            // at most 32 (more overflows): each half sorts 16 slots with a
            // register network; then the half-0 thread merges the two sorted
            // runs forward into ranks 0..15 and the half-1 thread backward
            // into ranks 31..16 (the keys are distinct: no ties to order),
            // and both write the exact leaves' output (or the list to
            // rescore)
            const int rtA = tid & 127, rtB = rtA | 128;  // the row's two threads
            const int ca = ccount[rtA], cb = ccount[rtB];
            const bool sel = row_ok && !rowflag[lr] && ca + cb <= 32;
            uint64_t* srt = reinterpret_cast<uint64_t*>(gsh);  // [2][16][128], minima are dead
            if (sel) {
                uint64_t v[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    const int u = 16 * half + e;
                    v[e] = u < ca ? cand[u * kTcThreads + rtA]
                                  : (u - ca < cb ? cand[(u - ca) * kTcThreads + rtB] : kKeyMax);
                }
                reg_bitonic_sort(v);
#pragma unroll
                for (int e = 0; e < 16; ++e) srt[(16 * half + e) * 128 + lr] = v[e];
            } else if (row_ok && half == 0 && !rowflag[lr]) {
                rowflag[lr] = 1;
                any_overflow = 1;
            }
            __syncthreads();
            uint64_t* rowlist = reinterpret_cast<uint64_t*>(cand);  // [32][128], the lists are dead
            if (sel) {
                const uint64_t* S0 = srt + lr;
                const uint64_t* S1 = srt + 16 * 128 + lr;
                uint64_t v[16];
                if (half == 0) {
                    int i = 0, j = 0;
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const uint64_t a = i < 16 ? S0[i * 128] : kKeyMax;
                        const uint64_t b = j < 16 ? S1[j * 128] : kKeyMax;
                        const bool ta = a <= b;
                        v[e] = ta ? a : b;
                        i += ta ? 1 : 0;
                        j += ta ? 0 : 1;
                    }
                } else {
                    int i = 15, j = 15;
#pragma unroll
                    for (int e = 15; e >= 0; --e) {
                        const uint64_t a = i >= 0 ? S0[i * 128] : 0ull;
                        const uint64_t b = j >= 0 ? S1[j * 128] : 0ull;
                        const bool ta = a > b;
                        v[e] = ta ? a : b;
                        i -= ta ? 1 : 0;
                        j -= ta ? 0 : 1;
                    }
                }
                const int r0s = 16 * half;  // rank of v[0]
                if (exact_leaf) {
                    const int gi = lid[iloc];
                    int32_t* oi = out_ids + ((int64_t)t * n + gi) * k;
                    float* od = out_d + ((int64_t)t * n + gi) * k;
                    if ((k & 3) == 0 && want == k && (((uintptr_t)out_ids | (uintptr_t)out_d) & 15) == 0) {
                        // whole rows of 16-byte groups (row starts are 16-byte
                        // aligned when k is a multiple of 4): four entries a store
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            if (r0s + e < want) {
                                int4 iv;
                                float4 dv4;
                                iv.x = lid[(uint32_t)v[e]];
                                iv.y = lid[(uint32_t)v[e + 1]];
                                iv.z = lid[(uint32_t)v[e + 2]];
                                iv.w = lid[(uint32_t)v[e + 3]];
                                dv4.x = unord_key((uint32_t)(v[e] >> 32));
                                dv4.y = unord_key((uint32_t)(v[e + 1] >> 32));
                                dv4.z = unord_key((uint32_t)(v[e + 2] >> 32));
                                dv4.w = unord_key((uint32_t)(v[e + 3] >> 32));
                                *reinterpret_cast<int4*>(oi + r0s + e) = iv;
                                *reinterpret_cast<float4*>(od + r0s + e) = dv4;
                            }
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (r0s + e < want) {
                                oi[r0s + e] = lid[(uint32_t)v[e]];
                                od[r0s + e] = unord_key((uint32_t)(v[e] >> 32));
                            }
                    }
                    if (half == 0)
                        for (int s2 = want; s2 < k; ++s2) {
                            oi[s2] = -1;
                            od[s2] = __int_as_float(0x7f800000);
                        }
                } else if (to_cands) {
                    uint16_t* oc = cand_out + (rowbase + iloc) * kp;
                    if ((kp & 3) == 0 && want == kp) {
                        // four local indices a store (row starts 8-byte aligned)
#pragma unroll
                        for (int e = 0; e < 16; e += 4)
                            if (r0s + e < want) {
                                uint2 u;
                                u.x = ((uint32_t)v[e] & 0xFFFFu) | ((uint32_t)v[e + 1] << 16);
                                u.y = ((uint32_t)v[e + 2] & 0xFFFFu) | ((uint32_t)v[e + 3] << 16);
                                *reinterpret_cast<uint2*>(oc + r0s + e) = u;
                            }
                    } else {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (r0s + e < want) oc[r0s + e] = (uint16_t)(uint32_t)v[e];
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (r0s + e < want) rowlist[(r0s + e) * 128 + lr] = v[e];
                }
            }
            __syncthreads();
            if (!exact_leaf && !to_cands) {
                // rescore the listed candidates of each row, one warp per row
                for (int rr = w; rr < 128; rr += kTcWarps) {
                    const int il2 = r0 + rr;
                    if (il2 >= m) break;
                    if (rowflag[rr]) continue;
                    const int gi = lid[il2];
                    leaf_rescore_list(L, lid, il2, rowlist + rr, 128, want, k, wsc + (size_t)kLeafWarpScratch * w,
                                      out_ids + ((int64_t)t * n + gi) * k, out_d + ((int64_t)t * n + gi) * k);
                }
            }
            __syncthreads();
        }
        if (any_overflow) {
            // warp-per-row path for the rows not done above
            const int ldD = G.ldD;
            for (int g0 = 0; g0 < 128 && r0 + g0 < m; g0 += G.RG) {
                if (32 * quad >= g0 && 32 * quad < g0 + G.RG) {
                    float* drow = Dblk + (size_t)(lr - g0) * ldD;
                    for (int c0 = 32 * half; c0 < Nm; c0 += 64) {
                        uint32_t r[32];
                        tc::tmem_ld32(trow + (uint32_t)c0, r);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int j = min(c0 + e, G.N_load - 1);
                            const float sdot = __uint_as_float(r[e]);
                            float dv;
                            if (PREC == 1) dv = ni + qn[j] - 2.f * sdot;
                            else dv = si * si * ni + qs[j] * qs[j] * qn[j] - 2.f * si * qs[j] * sdot;
                            drow[c0 + e] = dv;
                        }
                    }
                }
                __syncthreads();
                for (int rr = w; rr < G.RG && g0 + rr < 128; rr += kTcWarps) {
                    const int il2 = r0 + g0 + rr;
                    if (il2 >= m) break;
                    if (!rowflag[g0 + rr]) continue;
                    const float* drow = Dblk + (size_t)rr * ldD;
                    const int gi = lid[il2];
                    if (to_cands)
                        leaf_row_cands<PER>([&](int j) { return drow[j]; }, m, il2, kw,
                                            wsc + (size_t)kLeafWarpScratch * w, cand_out + (rowbase + il2) * kp);
                    else
                        leaf_row_finish<PER, kDT>(L, [&](int j) { return drow[j]; }, m, il2, lid, k, kw,
                                                  wsc + (size_t)kLeafWarpScratch * w,
                                                  out_ids + ((int64_t)t * n + gi) * k,
                                                  out_d + ((int64_t)t * n + gi) * k, !exact_leaf);
                }
                __syncthreads();
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (w == 0) tc::tmem_dealloc(tbase, ncols);
}

template <int PREC, int PER, int kDT>
static cudaError_t launch_tc(const CUtensorMap& map, const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                             const int32_t* perm, const float* qn, const float* qs, const uint8_t* qx, int k, int kp,
                             const TcGeom& G, int32_t* ids, float* dists, int* err, int* all_exact,
                             uint16_t* cand, uint8_t* leaf_flag, cudaStream_t st)
{
    auto kern = leaf_tc_kernel<PREC, PER, kDT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G.smem);
    if (e != cudaSuccess) return e;
    RowLoader<kDT> rl{x.X, x.ld, x.d, x.vec};
    const int nleaves = (int)P.leaf_off.size() - 1;
    const int RB = (P.max_leaf + 127) / 128;
    kern<<<dim3(nleaves * RB, T), kTcThreads, G.smem, st>>>(map, rl, x.n, perm, dp.leaf_off, nleaves, qn, qs, qx, k, kp,
                                                            G, ids, dists, err, all_exact, cand, leaf_flag);
    note_launches(1);
    return cudaGetLastError();
}

template <int PREC, int kDT>
static cudaError_t dispatch_tc(const CUtensorMap& map, const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                               const int32_t* perm, const float* qn, const float* qs, const uint8_t* qx, int k, int kp,
                               const TcGeom& G, int32_t* ids, float* dists, int* err, int* all_exact, uint16_t* cand,
                               uint8_t* leaf_flag, cudaStream_t st)
{
    // keys per lane in the row selection: leaves of up to 32 * PER points
    if (P.max_leaf <= 128)
        return launch_tc<PREC, 4, kDT>(map, x, P, dp, T, perm, qn, qs, qx, k, kp, G, ids, dists, err, all_exact, cand,
                                       leaf_flag, st);
    if (P.max_leaf <= 256)
        return launch_tc<PREC, 8, kDT>(map, x, P, dp, T, perm, qn, qs, qx, k, kp, G, ids, dists, err, all_exact, cand,
                                       leaf_flag, st);
    return launch_tc<PREC, 16, kDT>(map, x, P, dp, T, perm, qn, qs, qx, k, kp, G, ids, dists, err, all_exact, cand,
                                    leaf_flag, st);
}

// Gather + quantise the leaf-ordered copy (or quantise the rows once in
// point order), then the leaf kernel, for one element type of X (explicitly
// instantiated per type).
// cand, leaf_flag (both or neither): candidates of the rows of leaves that
// are not exact, for run_leaf_rescore_staged, and each leaf's exactness.
template <int kDT>
cudaError_t leaf_tc_run(int prec, const CUtensorMap& map, const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                        const int32_t* perm, int dq, void* Xq, float* qn, float* qs, uint8_t* qx, int k, int kp,
                        const TcGeom& G, int32_t* ids, float* dists, int* err, int* all_exact, uint16_t* cand,
                        uint8_t* leaf_flag, cudaStream_t st)
{
    // G.xg set: one quantised copy in point order (the leaf kernel gathers
    // the leaves' rows itself), else a leaf-ordered copy per tree
    const bool by_point = G.xg != nullptr;
    const int64_t rows = by_point ? x.n : (int64_t)T * x.n;
    const int32_t* gperm = by_point ? nullptr : perm;
    const int gblocks = (int)std::min<int64_t>((rows + 7) / 8, (int64_t)num_sms() * 16);
    RowLoader<kDT> rl{x.X, x.ld, x.d, x.vec};
    const RowLoader<kDtU8> rb{x.Xb, x.ldb, x.d, true};
    // byte input laid out for 16-byte row loads
    const bool u8_aligned =
        x.dtype == kDtU8 && ((uintptr_t)x.X % 16 == 0) && (x.ld % 16 == 0) && (x.d % 16 == 0);
    if (prec == 1)
        gather_quant_kernel<1, kDT><<<gblocks, 256, 0, st>>>(rl, rb, x.xb_bad, rows, gperm, dq, Xq, qn, qs, qx,
                                                             u8_aligned);
    else
        gather_quant_kernel<2, kDT><<<gblocks, 256, 0, st>>>(rl, rb, x.xb_bad, rows, gperm, dq, Xq, qn, qs, qx,
                                                             u8_aligned);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (prec == 1)
        return dispatch_tc<1, kDT>(map, x, P, dp, T, perm, qn, qs, qx, k, kp, G, ids, dists, err, all_exact, cand,
                                   leaf_flag, st);
    return dispatch_tc<2, kDT>(map, x, P, dp, T, perm, qn, qs, qx, k, kp, G, ids, dists, err, all_exact, cand,
                               leaf_flag, st);
}

}  // namespace knng
