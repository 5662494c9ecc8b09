// FP32 rescoring of the reduced-precision leaf candidates (the leaf graphs of
// Sec. 3.1 of arXiv:1307.7852 with a BF16 / FP8 candidate stage), one CTA per
// (tree, leaf).
//
// The tensor-core leaf kernel leaves, for every row of a leaf that is not
// exact in reduced precision, its k' candidates (local indices in the leaf).
// Rescoring them with the canonical FP32 distance reads k' rows of d floats
// per point; fetched one pair at a time from L2 that is k' * d * 4 bytes per
// point (0.6 TB over the eight trees of a 1M x 960 build).  Here the leaf's
// rows stream through shared memory instead, in 32-entry slices (one block
// of the canonical distance), double-buffered with cp.async, so each row of
// the leaf crosses L2 once per tree:
//   * one thread per row holds its own slice in registers and one running
//     sum per candidate; per slice it forms the eight 4-entry partials of
//     every candidate pair, closes the block by the butterfly and adds it to
//     the pair's sum -- exactly the canonical distance, block by block;
//   * thread r reads the slice's eight 16-byte columns in the order
//     u ^ (r mod 8), so the eight threads of a quarter warp touch eight
//     different bank groups whatever rows they read;
//   * at the end every row keeps its k best by (distance, id).
// Leaves that are exact in reduced precision (their lists are final) are
// skipped by a flag the leaf kernel writes.
#include "knng_common.cuh"
#include "knng_internal.h"

namespace knng {

namespace {
constexpr int kSlice = 32;       // floats per row and slice (one block of the distance)
constexpr int kMaxCand = 40;     // candidates per row handled here
}  // namespace

// Canonical block value of a pair: own slice a (columns in the order
// u ^ x, u = 0..7, already in registers), candidate slice b in shared
// memory.  s[u] is the partial of column u ^ x; since the block's butterfly
// pairs columns by xor (q with q ^ 4, then q ^ 2, then q ^ 1), relabelling
// them by xor with x only swaps the operands of some additions, so the tree
// below over s[] gives the block value bit for bit -- and, t = a - b and
// b - a squaring alike, the same value whichever row is the own one.
// (Scalar FP32: packed pairs need their operands in adjacent registers,
// which these columns are not, and measured slower.)
__device__ __forceinline__ float slice_block(const float4 (&a)[8], const float4* __restrict__ b, int x)
{
    float s[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const float4 v = b[u ^ x];
        float acc = 0.f, t;
        t = a[u].x - v.x; acc = fmaf(t, t, acc);
        t = a[u].y - v.y; acc = fmaf(t, t, acc);
        t = a[u].z - v.z; acc = fmaf(t, t, acc);
        t = a[u].w - v.w; acc = fmaf(t, t, acc);
        s[u] = acc;
    }
    return ((s[0] + s[4]) + (s[2] + s[6])) + ((s[1] + s[5]) + (s[3] + s[7]));
}

// grid (nleaves, T); blockDim >= the largest leaf (multiple of 32, <= 512).
// cand: [T * n][kp] local indices (u16) of every row's candidates, the first
// want = min(kp, m - 1) valid.  X rows: FP32, 16-byte aligned, ld % 4 == 0.
//
// A pair listed by both of its rows (r in c's list and c in r's) is scored
// once, by the smaller row: the canonical distance is symmetric bit for bit,
// so the other row takes the value from a table in shared memory.
// Membership is a 512-bit bitmap per row.  (Dealing the pairs out evenly,
// both rows then read from shared memory, measured slower: the row-per-
// thread form keeps the own slice in registers.)
template <int KC>
__global__ void __launch_bounds__(512, 1) leaf_rescore_staged_kernel(
    const float* __restrict__ X, int64_t ld, int d, int64_t n, const int32_t* __restrict__ perm,
    const int32_t* __restrict__ leaf_off, int nleaves, const uint8_t* __restrict__ leaf_exact,
    const uint16_t* __restrict__ cand, int kp, int k, int32_t* __restrict__ out_ids, float* __restrict__ out_d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int t = blockIdx.y, leaf = blockIdx.x;
    if (leaf_exact[(int64_t)t * nleaves + leaf]) return;
    const int off = leaf_off[leaf];
    const int m = leaf_off[leaf + 1] - off;
    const int mp = (m + 7) & ~7;
    // [2][mp][8] float4 slices | lid[mp] | bits[mp][16] u32 | cand_s[mp][kp] u16
    float4* buf = reinterpret_cast<float4*>(smem_raw);
    int32_t* lid = reinterpret_cast<int32_t*>(buf + 2 * (size_t)mp * 8);
    uint32_t* bits = reinterpret_cast<uint32_t*>(lid + mp);
    uint16_t* cand_s = reinterpret_cast<uint16_t*>(bits + (size_t)mp * 16);
    float* res = reinterpret_cast<float*>(buf);  // [mp][kp], after the slices
    const int tid = threadIdx.x;
    const int64_t rowbase = (int64_t)t * n + off;
    for (int j = tid; j < m; j += blockDim.x) lid[j] = perm[rowbase + j];

    const bool active = tid < m;
    const int want = min(kp, m - 1);
    uint16_t c[KC];
    float tot[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) {
        c[i] = 0;
        tot[i] = 0.f;
    }
    if (active) {
        const uint16_t* cr = cand + (rowbase + tid) * kp;
        uint32_t* mybits = bits + (size_t)tid * 16;  // this row's bitmap: only this thread writes it
#pragma unroll
        for (int z = 0; z < 16; ++z) mybits[z] = 0u;
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (i < want) {
                c[i] = cr[i];
                cand_s[(size_t)tid * kp + i] = c[i];
                mybits[c[i] >> 5] |= 1u << (c[i] & 31);
            }
    }
    __syncthreads();
    // the pairs this row scores: its candidate is larger, or does not list it
    uint64_t mine = 0ull;
    if (active) {
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (i < want) {
                const int cc = c[i];
                const bool listed = (bits[(size_t)cc * 16 + (tid >> 5)] >> (tid & 31)) & 1u;
                if (cc > tid || !listed) mine |= 1ull << i;
            }
    }

    const int nslices = (d + kSlice - 1) / kSlice;
    auto stage = [&](int sl, int b) {
        float4* dst = buf + (size_t)b * mp * 8;
        for (int u = tid; u < m * 8; u += blockDim.x) {
            const int r = u >> 3, col = u & 7;
            const int j = sl * kSlice + 4 * col;
            const int avail = d - j;
            const float* src = X + (uint64_t)(uint32_t)lid[r] * (uint64_t)ld;
            const int bytes = avail >= 4 ? 16 : (avail > 0 ? 4 * avail : 0);
            cp_async16(dst + (size_t)r * 8 + col, bytes > 0 ? src + j : src, bytes);
        }
        cp_async_commit();
    };
    const int x8 = tid & 7;  // columns read in the order u ^ x8: a quarter warp hits eight bank groups

    stage(0, 0);
    for (int sl = 0; sl < nslices; ++sl) {
        if (sl + 1 < nslices) {
            stage(sl + 1, (sl + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (active) {
            const float4* B = buf + (size_t)(sl & 1) * mp * 8;
            float4 a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = B[(size_t)tid * 8 + (u ^ x8)];
#pragma unroll
            for (int i = 0; i < KC; ++i)
                if ((mine >> i) & 1ull) tot[i] = tot[i] + slice_block(a, B + (size_t)c[i] * 8, x8);
        }
        __syncthreads();  // the buffer of this slice is staged again two slices on
    }
    // exchange: every row publishes what it scored, then takes the pairs its
    // candidate scored from the candidate's row of the table
    if (active) {
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if ((mine >> i) & 1ull) res[(size_t)tid * kp + i] = tot[i];
    }
    __syncthreads();
    if (!active) return;
#pragma unroll
    for (int i = 0; i < KC; ++i)
        if (i < want && !((mine >> i) & 1ull)) {
            const int cc = c[i];
            const uint16_t* lc = cand_s + (size_t)cc * kp;
            int j = 0;
            while (j < kp - 1 && lc[j] != (uint16_t)tid) ++j;
            tot[i] = res[(size_t)cc * kp + j];
        }
    // the k best of the row's candidates by (distance, point id)
    uint64_t key[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) key[i] = i < want ? pack_key(tot[i], (uint32_t)lid[c[i]]) : kKeyMax;
    const int gi = lid[tid];
    int32_t* oi = out_ids + ((int64_t)t * n + gi) * k;
    float* od = out_d + ((int64_t)t * n + gi) * k;
    // entries two at a time (8-byte stores: k is even and the row starts
    // 8-byte aligned), else one at a time
    const bool pairs2 = (k & 1) == 0 && (((uintptr_t)out_ids | (uintptr_t)out_d) & 7) == 0;
    uint64_t prev = 0;
    int32_t id_lo = -1;
    float d_lo = 0.f;
    for (int s = 0; s < k; ++s) {
        uint64_t best = kKeyMax;
#pragma unroll
        for (int i = 0; i < KC; ++i)
            if (key[i] < best && (s == 0 || key[i] > prev)) best = key[i];
        const bool ok = s < want && best != kKeyMax;
        const int32_t id = ok ? (int32_t)(uint32_t)best : -1;
        const float dv = ok ? unord_key((uint32_t)(best >> 32)) : __int_as_float(0x7f800000);
        if (!pairs2) {
            oi[s] = id;
            od[s] = dv;
        } else if (s & 1) {
            *reinterpret_cast<int2*>(oi + s - 1) = make_int2(id_lo, id);
            *reinterpret_cast<float2*>(od + s - 1) = make_float2(d_lo, dv);
        } else {
            id_lo = id;
            d_lo = dv;
        }
        prev = best;
    }
}

static size_t staged_smem(int max_leaf, int kp)
{
    const size_t mp = (size_t)((max_leaf + 7) & ~7);
    return 2 * mp * 8 * sizeof(float4) + mp * sizeof(int32_t) + mp * 16 * sizeof(uint32_t) +
           mp * kp * sizeof(uint16_t);
}

bool leaf_rescore_staged_ok(const XDesc& x, int kp, int max_leaf)
{
    return x.dtype == kDtF32 && x.vec && (x.ld % 4) == 0 && kp <= kMaxCand && max_leaf <= 512 &&
           staged_smem(max_leaf, kp) <= 220 * 1024;
}

cudaError_t run_leaf_rescore_staged(const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                                    const int32_t* perm, const uint8_t* leaf_exact, const uint16_t* cand, int kp,
                                    int k, int32_t* ids, float* dists, cudaStream_t st)
{
    const int nleaves = (int)P.leaf_off.size() - 1;
    const int threads = std::max(32, (P.max_leaf + 31) & ~31);
    const size_t smem = staged_smem(P.max_leaf, kp);
    // candidate capacity per row: the smallest of 16, 24, 32, 40 holding k'
    auto kern = kp <= 16 ? leaf_rescore_staged_kernel<16>
              : kp <= 24 ? leaf_rescore_staged_kernel<24>
              : kp <= 32 ? leaf_rescore_staged_kernel<32>
                         : leaf_rescore_staged_kernel<40>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(nleaves, T), threads, smem, st>>>(static_cast<const float*>(x.X), x.ld, x.d, x.n, perm, dp.leaf_off,
                                                  nleaves, leaf_exact, cand, kp, k, ids, dists);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace knng
