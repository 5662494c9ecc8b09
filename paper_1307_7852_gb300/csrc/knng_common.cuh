// Device-side building blocks shared by the kernels of the library:
// Philox4x32-10, the order-preserving float key, row loads, the canonical
// FP32 squared distance, and warp-level selection and sorting.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define KNNG_FULL_MASK 0xFFFFFFFFu

namespace knng {

constexpr uint64_t kKeyMax = ~0ull;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments
// 0x9E3779B9 / 0xBB67AE85.
// ---------------------------------------------------------------------------
__host__ __device__ inline uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Triangular direction entry from one Philox word: (lo16 + hi16 - 65535)/2^16.
__host__ __device__ inline float tri_entry(uint32_t u)
{
    return (float)((int32_t)(u & 0xFFFFu) + (int32_t)(u >> 16) - 65535) * (1.0f / 65536.0f);
}

// Order-preserving map of FP32 bits to u32: sign clear -> set sign bit;
// sign set -> invert all bits.  -0 orders just below +0.
__device__ __forceinline__ uint32_t ord_key(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float unord_key(uint32_t o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}
__device__ __forceinline__ uint64_t pack_key(float dist, uint32_t id)
{
    return ((uint64_t)ord_key(dist) << 32) | id;
}

// Asynchronous global-to-shared copies (cp.async): 16 bytes (zero-filled past
// src_bytes) or 4 bytes; completion by commit groups.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int src_bytes)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------------------
// Row loads.  Point i of X starts at element i*ld; d entries.  load4 returns
// entries j..j+3 (zero past d) widened to FP32.  Element types: FP32, FP16
// and unsigned bytes (byte values widen exactly, so every FP32 computation
// on them is the one on the equal float rows).
// ---------------------------------------------------------------------------
constexpr int kDtF32 = 0, kDtF16 = 1, kDtU8 = 2;

__device__ __forceinline__ float4 bytes_to_float4(uint32_t u)
{
    return make_float4((float)(u & 0xFFu), (float)((u >> 8) & 0xFFu), (float)((u >> 16) & 0xFFu),
                       (float)(u >> 24));
}

template <int kDT>
struct RowLoader {
    const void* X;
    int64_t ld;
    int d;
    bool vec;  // rows 16-byte (F32) / 8-byte (F16) / 4-byte (U8) aligned and ld multiple of 4

    // element offset of row i (ids < 2^31, ld < 2^31: one 32x32->64 multiply)
    __device__ __forceinline__ uint64_t row_off(int64_t i) const
    {
        return (uint64_t)(uint32_t)i * (uint32_t)ld;
    }

    __device__ __forceinline__ float4 load4(int64_t i, int j) const
    {
        float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kDT == kDtF16) {
            const __half* row = static_cast<const __half*>(X) + row_off(i);
            if (vec && j + 3 < d) {
                const uint2 u = __ldg(reinterpret_cast<const uint2*>(row + j));
                const __half2 a = *reinterpret_cast<const __half2*>(&u.x);
                const __half2 b = *reinterpret_cast<const __half2*>(&u.y);
                const float2 fa = __half22float2(a), fb = __half22float2(b);
                r = make_float4(fa.x, fa.y, fb.x, fb.y);
            } else {
                if (j + 0 < d) r.x = __half2float(row[j + 0]);
                if (j + 1 < d) r.y = __half2float(row[j + 1]);
                if (j + 2 < d) r.z = __half2float(row[j + 2]);
                if (j + 3 < d) r.w = __half2float(row[j + 3]);
            }
        } else if (kDT == kDtU8) {
            const uint8_t* row = static_cast<const uint8_t*>(X) + row_off(i);
            if (vec && j + 3 < d) {
                r = bytes_to_float4(__ldg(reinterpret_cast<const unsigned int*>(row + j)));
            } else {
                if (j + 0 < d) r.x = (float)__ldg(row + j + 0);
                if (j + 1 < d) r.y = (float)__ldg(row + j + 1);
                if (j + 2 < d) r.z = (float)__ldg(row + j + 2);
                if (j + 3 < d) r.w = (float)__ldg(row + j + 3);
            }
        } else {
            const float* row = static_cast<const float*>(X) + row_off(i);
            if (vec && j + 3 < d) {
                r = __ldg(reinterpret_cast<const float4*>(row + j));
            } else {
                if (j + 0 < d) r.x = __ldg(row + j + 0);
                if (j + 1 < d) r.y = __ldg(row + j + 1);
                if (j + 2 < d) r.z = __ldg(row + j + 2);
                if (j + 3 < d) r.w = __ldg(row + j + 3);
            }
        }
        return r;
    }
    // entries j..j+3 of row i when rows are vector-aligned and j + 3 < d
    __device__ __forceinline__ float4 load4v(int64_t i, int j) const
    {
        if (kDT == kDtF16) {
            const uint2 u = __ldg(reinterpret_cast<const uint2*>(static_cast<const __half*>(X) + row_off(i) + j));
            const float2 fa = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
            const float2 fb = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
            return make_float4(fa.x, fa.y, fb.x, fb.y);
        }
        if (kDT == kDtU8) return bytes_to_float4(load_u8x4(i, j));
        return __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(X) + row_off(i) + j));
    }
    // bytes j..j+3 of row i packed little-endian (U8 rows, vector-aligned)
    __device__ __forceinline__ uint32_t load_u8x4(int64_t i, int j) const
    {
        return __ldg(reinterpret_cast<const unsigned int*>(static_cast<const uint8_t*>(X) + row_off(i) + j));
    }
    // every load of a row is a full vector load (aligned rows, d % 4 == 0)
    __device__ __forceinline__ bool all_vec() const { return vec && (d & 3) == 0; }
    // byte rows whose squared distances stay below 2^24 (d * 255^2 < 2^24):
    // every partial sum of the canonical FP32 distance is then an exact
    // integer, so integer arithmetic in any order gives the same value
    __device__ __forceinline__ bool int_exact() const { return kDT == kDtU8 && d <= 256; }

    // L2 prefetch of row i, one 128-byte line per lane (the lines that hold
    // the row's d entries only)
    __device__ __forceinline__ void prefetch_l2(int64_t i, int lane) const
    {
        constexpr int es = kDT == kDtF16 ? 2 : kDT == kDtU8 ? 1 : 4;
        const char* row = static_cast<const char*>(X) + row_off(i) * es;
        const uintptr_t first = (uintptr_t)row & ~(uintptr_t)127;
        const uintptr_t end = (uintptr_t)row + (uintptr_t)d * es;
        for (uintptr_t a = first + 128 * (uintptr_t)lane; a < end; a += 4096)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a < (uintptr_t)row ? (uintptr_t)row : a));
    }

    __device__ __forceinline__ float load1(int64_t i, int j) const
    {
        if (kDT == kDtF16) return __half2float(static_cast<const __half*>(X)[row_off(i) + j]);
        if (kDT == kDtU8) return (float)__ldg(static_cast<const uint8_t*>(X) + row_off(i) + j);
        return __ldg(static_cast<const float*>(X) + row_off(i) + j);
    }
};

// ---------------------------------------------------------------------------
// Canonical FP32 squared distance.  The entries are cut into blocks of 32:
// in block b, partial q = 0..7 sums s_q = fmaf(t, t, s_q), t = x_a[j] - x_b[j],
// over j = 32b + 4q + e (e = 0..3); the block's value is the xor butterfly of
// its eight partials, B_b = ((s0 + s4) + (s2 + s6)) + ((s1 + s5) + (s3 + s7)),
// and the distance adds B_0, B_1, ... in block order.  Every term is
// non-negative, so the relative error stays below (8 + ceil(d/32)) * 2^-24
// (8.1e-6 at d = 4096), and the value depends only on the two rows, so
// D(a, b) == D(b, a) bit for bit.  Because each block is closed before the
// next, a kernel can stream the rows in 32-entry slices and keep one running
// sum per pair.
//
// The warp form: lane l holds entries 128c + 4l .. +3 of 128-entry chunk c,
// which are partial l & 7 of block 4c + (l >> 3); a butterfly over the eight
// lanes of each group closes the four blocks, and their values are added in
// order.  Entries past d load as 0 and add nothing (fmaf(0, 0, s) = s, and a
// block of zeros adds +0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float chunk_blocks_add(float tot, float blk)
{
    // blk: lane group g holds block 4c + g; add the four in block order
    const float b0 = __shfl_sync(KNNG_FULL_MASK, blk, 0);
    const float b1 = __shfl_sync(KNNG_FULL_MASK, blk, 8);
    const float b2 = __shfl_sync(KNNG_FULL_MASK, blk, 16);
    const float b3 = __shfl_sync(KNNG_FULL_MASK, blk, 24);
    return (((tot + b0) + b1) + b2) + b3;
}

template <int kDT>
__device__ __forceinline__ float warp_canon_dist(const RowLoader<kDT>& L, int64_t a, int64_t b)
{
    const int lane = threadIdx.x & 31;
    float tot = 0.0f;
    for (int j0 = 0; j0 < L.d; j0 += 128) {
        const int j = j0 + 4 * lane;
        float s = 0.0f;
        if (j < L.d) {
            const float4 xa = L.load4(a, j), xb = L.load4(b, j);
            float t;
            t = xa.x - xb.x; s = fmaf(t, t, s);
            t = xa.y - xb.y; s = fmaf(t, t, s);
            t = xa.z - xb.z; s = fmaf(t, t, s);
            t = xa.w - xb.w; s = fmaf(t, t, s);
        }
        s += __shfl_xor_sync(KNNG_FULL_MASK, s, 4);
        s += __shfl_xor_sync(KNNG_FULL_MASK, s, 2);
        s += __shfl_xor_sync(KNNG_FULL_MASK, s, 1);
        tot = chunk_blocks_add(tot, s);
    }
    return tot;
}

// ---------------------------------------------------------------------------
// Warp bitonic sort of 32*E 64-bit keys, E per lane; element index
// i = lane*E + e.  Ascending on return.
// ---------------------------------------------------------------------------
template <int E>
__device__ __forceinline__ void warp_bitonic_sort(uint64_t (&v)[E])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int kk = 2; kk <= 32 * E; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j >= E) {
                const int lj = j / E;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int i = lane * E + e;
                    const uint64_t other = __shfl_xor_sync(KNNG_FULL_MASK, v[e], lj);
                    const bool up = (i & kk) == 0;
                    const bool lower = (i & j) == 0;
                    const bool keep_min = (lower == up);
                    const uint64_t mn = v[e] < other ? v[e] : other;
                    const uint64_t mx = v[e] < other ? other : v[e];
                    v[e] = keep_min ? mn : mx;
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int p = e ^ j;
                    if (p > e) {
                        const int i = lane * E + e;
                        const bool up = (i & kk) == 0;
                        const uint64_t a = v[e], b = v[p];
                        const bool sw = up ? (a > b) : (a < b);
                        v[e] = sw ? b : a;
                        v[p] = sw ? a : b;
                    }
                }
            }
        }
    }
}

// The same network on 32-bit values.
template <int E>
__device__ __forceinline__ void warp_bitonic_sort32(uint32_t (&v)[E])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int kk = 2; kk <= 32 * E; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j >= E) {
                const int lj = j / E;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int i = lane * E + e;
                    const uint32_t other = __shfl_xor_sync(KNNG_FULL_MASK, v[e], lj);
                    const bool keep_min = ((i & j) == 0) == ((i & kk) == 0);
                    v[e] = keep_min ? min(v[e], other) : max(v[e], other);
                }
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int p = e ^ j;
                    if (p > e) {
                        const int i = lane * E + e;
                        const bool up = (i & kk) == 0;
                        const uint32_t lo = min(v[e], v[p]), hi = max(v[e], v[p]);
                        v[e] = up ? lo : hi;
                        v[p] = up ? hi : lo;
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// Warp radix select.  Among cnt unique 64-bit keys key(idx), idx in [0, cnt),
// returns the threshold K such that exactly min(want, cnt) keys are <= K
// (want >= 1).  The bits that all keys share (from their minimum and
// maximum) are skipped; the rest is resolved 8 bits per pass from the most
// significant end, and a pass ends the search as soon as every key that
// matches the prefix must be taken.  hist: 256 words of shared memory private
// to the warp; lane l owns bins l, l+32, ..., l+224 (conflict-free).
// Collective: all 32 lanes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t lowmask64(int b)
{
    return b >= 64 ? ~0ull : ((1ull << b) - 1ull);
}

template <class KeyFn>
__device__ uint64_t warp_select_threshold(const KeyFn& key, int cnt, int want, uint32_t* hist)
{
    if (want >= cnt) return kKeyMax;
    const int lane = threadIdx.x & 31;
    uint64_t mn = kKeyMax, mx = 0;
    for (int idx = lane; idx < cnt; idx += 32) {
        const uint64_t kv = key(idx);
        mn = kv < mn ? kv : mn;
        mx = kv > mx ? kv : mx;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const uint64_t a = __shfl_xor_sync(KNNG_FULL_MASK, mn, o);
        const uint64_t b = __shfl_xor_sync(KNNG_FULL_MASK, mx, o);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
    }
    int hi = 64 - __clzll((long long)(mn ^ mx));  // bits [hi, 64) are common (cnt >= 2)
    uint64_t mask = ~lowmask64(hi);
    uint64_t prefix = mn & mask;
    int rank = want;
    while (true) {
        const int lo = hi > 8 ? hi - 8 : 0;
        const uint32_t dmask = (uint32_t)lowmask64(hi - lo);
#pragma unroll
        for (int b = 0; b < 8; ++b) hist[b * 32 + lane] = 0;
        __syncwarp();
        for (int idx = lane; idx < cnt; idx += 32) {
            const uint64_t kv = key(idx);
            if ((kv & mask) == prefix) atomicAdd(&hist[(uint32_t)(kv >> lo) & dmask], 1u);
        }
        __syncwarp();
        uint32_t c[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) c[b] = hist[b * 32 + lane];
        // the 32-bin chunk in which the rank falls, then the bin inside it
        uint32_t run = 0, before_chunk = 0, mine = 0;
        int chunk = 0;
        bool found = false;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint32_t tot = __reduce_add_sync(KNNG_FULL_MASK, c[b]);
            if (!found && run < (uint32_t)rank && (uint32_t)rank <= run + tot) {
                found = true;
                chunk = b;
                before_chunk = run;
                mine = c[b];
            }
            run += tot;
        }
        uint32_t incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(KNNG_FULL_MASK, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t excl = incl - mine;
        const bool own = before_chunk + excl < (uint32_t)rank && (uint32_t)rank <= before_chunk + incl;
        const int owner = __ffs(__ballot_sync(KNNG_FULL_MASK, own)) - 1;
        const uint32_t digit = (uint32_t)(chunk * 32 + owner);
        const uint32_t before = before_chunk + __shfl_sync(KNNG_FULL_MASK, excl, owner);
        const uint32_t inbin = __shfl_sync(KNNG_FULL_MASK, mine, owner);
        prefix |= (uint64_t)digit << lo;
        mask |= (uint64_t)dmask << lo;
        rank -= (int)before;
        __syncwarp();
        if ((uint32_t)rank == inbin || lo == 0) return prefix | lowmask64(lo);
        hi = lo;
    }
}

// Writes the indices of the keys <= thr, in index order, to out[] (shared or
// global memory); returns their count.  Collective: all 32 lanes.
template <class KeyFn>
__device__ int warp_compact_le(const KeyFn& key, int cnt, uint64_t thr, int* out)
{
    const int lane = threadIdx.x & 31;
    int base = 0;
    for (int it = 0; it < cnt; it += 32) {
        const int idx = it + lane;
        const bool sel = idx < cnt && key(idx) <= thr;
        const uint32_t b = __ballot_sync(KNNG_FULL_MASK, sel);
        if (sel) out[base + __popc(b & lanemask_lt())] = idx;
        base += __popc(b);
    }
    return base;
}

// Open-addressing set of point ids in shared memory (EMPTY = -1), linear
// probing, multiplicative hash on the high bits.  Returns true if id was not
// yet present.  The caller sizes the table above the number of insertions,
// so the probe loop always finds a free slot or the id.
__device__ __forceinline__ bool hash_insert(int* tab, uint32_t hshift, uint32_t hmask, int id)
{
    uint32_t h = ((uint32_t)id * 0x9E3779B1u) >> hshift;
    while (true) {
        const int old = atomicCAS(&tab[h], -1, id);
        if (old == -1) return true;
        if (old == id) return false;
        h = (h + 1) & hmask;
    }
}

}  // namespace knng

namespace knng {

// Sorted `want` smallest (want <= 64) of cnt unique keys key(0..cnt)
// (cnt <= 32*PER), written ascending to out[0..min(want, cnt)) in shared
// memory; returns that count.  The want-th smallest distance part (high 32
// bits) among the lane minima (or, for want > 32, among every lane's two
// smallest keys) bounds the answer from above: the keys whose distance part
// is at most that value contain it.  Usually few do: up to 32 are ranked by
// counting, up to 128 sorted by a small bitonic network; otherwise the radix
// select decides.
// scratch: >= 128 keys, hist: 256 words, both private to the warp.
template <int PER, class KeyFn>
__device__ int warp_topk_sorted(const KeyFn& key, int cnt, int want, uint64_t* out, uint64_t* scratch,
                                uint32_t* hist)
{
    const int lane = threadIdx.x & 31;
    if (want > cnt) want = cnt;
    if (want <= 0) return 0;
    uint64_t x[PER];
    // distance parts (high 32 bits) of each lane's two smallest keys
    uint32_t a = 0xFFFFFFFFu, b = 0xFFFFFFFFu;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int idx = lane + 32 * e;
        x[e] = idx < cnt ? key(idx) : kKeyMax;
        const uint32_t h = (uint32_t)(x[e] >> 32);
        if (h < a) { b = a; a = h; }
        else if (h < b) b = h;
    }
    // tau: the want-th smallest of those distance parts.  At least `want`
    // keys have a distance part <= tau, so every key of the answer does too.
    const int wi = want - 1;
    uint32_t tau;
    if (want <= 32) {
        uint32_t s1[1] = {a};
        warp_bitonic_sort32<1>(s1);
        tau = __shfl_sync(KNNG_FULL_MASK, s1[0], wi);
    } else {
        uint32_t s2[2] = {a, b};
        warp_bitonic_sort32<2>(s2);
        tau = __shfl_sync(KNNG_FULL_MASK, (wi & 1) ? s2[1] : s2[0], wi >> 1);
    }
    int c = 0;
#pragma unroll
    for (int e = 0; e < PER; ++e) c += __popc(__ballot_sync(KNNG_FULL_MASK, (uint32_t)(x[e] >> 32) <= tau));
    if (c <= 128) {
        int base = 0;
#pragma unroll
        for (int e = 0; e < PER; ++e) {
            const bool sel = (uint32_t)(x[e] >> 32) <= tau;
            const uint32_t bl = __ballot_sync(KNNG_FULL_MASK, sel);
            if (sel) scratch[base + __popc(bl & lanemask_lt())] = x[e];
            base += __popc(bl);
        }
        __syncwarp();
        if (c <= 32) {
            // rank by counting (position breaks equal keys, so ranks differ)
            const uint64_t v = lane < c ? scratch[lane] : kKeyMax;
            int rank = 0;
            for (int j = 0; j < c; ++j) {
                const uint64_t y = scratch[j];
                rank += (y < v || (y == v && j < lane)) ? 1 : 0;
            }
            if (lane < c && rank < want) out[rank] = v;
        } else if (c <= 64) {
            uint64_t v[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) v[e] = lane * 2 + e < c ? scratch[lane * 2 + e] : kKeyMax;
            warp_bitonic_sort<2>(v);
#pragma unroll
            for (int e = 0; e < 2; ++e)
                if (lane * 2 + e < want) out[lane * 2 + e] = v[e];
        } else {
            uint64_t v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = lane * 4 + e < c ? scratch[lane * 4 + e] : kKeyMax;
            warp_bitonic_sort<4>(v);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (lane * 4 + e < want) out[lane * 4 + e] = v[e];
        }
    } else {
        auto kx = [&](int idx) -> uint64_t { return key(idx); };
        const uint64_t thr = warp_select_threshold(kx, cnt, want, hist);
        int base = 0;
        for (int it = 0; it < cnt; it += 32) {
            const int idx = it + lane;
            const uint64_t kv = idx < cnt ? key(idx) : kKeyMax;
            const bool sel = idx < cnt && kv <= thr;
            const uint32_t bl = __ballot_sync(KNNG_FULL_MASK, sel);
            if (sel) scratch[base + __popc(bl & lanemask_lt())] = kv;
            base += __popc(bl);
        }
        __syncwarp();
        uint64_t v[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) v[e] = lane * 2 + e < want ? scratch[lane * 2 + e] : kKeyMax;
        warp_bitonic_sort<2>(v);
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (lane * 2 + e < want) out[lane * 2 + e] = v[e];
    }
    __syncwarp();
    return want;
}

// Canonical distances from point a to W points b[0..W) (W = 8, 16 or 32;
// b in shared memory, entries c >= nb unused); lane l returns the distance to
// b[l % W] (for l % W < nb).  Rows must be vector-aligned with d % 4 == 0.
// Per 128-entry chunk each lane forms its partials (entries 128c + 4l + e,
// fmaf) for the W points; recursive halving over the eight lanes of each
// group (offsets 4, 2, 1: each lane keeps half of its values and receives
// its partner's copy of them) performs the additions of the block butterfly
// and leaves lane l with the block values of points (W/8)(l & 7) + i,
// i < W/8, for block 4c + (l >> 3); the four blocks are then added in order
// to running sums.  Bit-identical to warp_canon_dist, with far fewer
// shuffles and W row loads in flight.
template <int W, int kDT>
__device__ __forceinline__ float warp_canon_dist_batch(const RowLoader<kDT>& L, int64_t a, const int* b, int nb)
{
    static_assert(W == 8 || W == 16 || W == 32, "batch of 8, 16 or 32 points");
    constexpr int V = W / 8;  // values a lane keeps after the halving
    const int lane = threadIdx.x & 31;
    const int g8 = lane & 7;
    int bid[W];
#pragma unroll
    for (int c = 0; c < W; ++c) bid[c] = c < nb ? b[c] : (int)a;
    float tot[V];
#pragma unroll
    for (int i = 0; i < V; ++i) tot[i] = 0.f;
    for (int j0 = 0; j0 < L.d; j0 += 128) {
        const int j = j0 + 4 * lane;
        float p[W];
#pragma unroll
        for (int c = 0; c < W; ++c) p[c] = 0.f;
        if (j < L.d) {
            const float4 xa = L.load4v(a, j);
#pragma unroll
            for (int c0 = 0; c0 < W; c0 += 8) {
                float4 xb[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) xb[c] = L.load4v(bid[c0 + c], j);
                // points c and c + 1 side by side in packed FP32 pairs (each
                // half rounds exactly like the scalar operation)
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    const float4 u = xb[c], v = xb[c + 1];
                    float2 acc = make_float2(0.f, 0.f), t;
                    t = __fadd2_rn(make_float2(xa.x, xa.x), make_float2(-u.x, -v.x)); acc = __ffma2_rn(t, t, acc);
                    t = __fadd2_rn(make_float2(xa.y, xa.y), make_float2(-u.y, -v.y)); acc = __ffma2_rn(t, t, acc);
                    t = __fadd2_rn(make_float2(xa.z, xa.z), make_float2(-u.z, -v.z)); acc = __ffma2_rn(t, t, acc);
                    t = __fadd2_rn(make_float2(xa.w, xa.w), make_float2(-u.w, -v.w)); acc = __ffma2_rn(t, t, acc);
                    p[c0 + c] = acc.x;
                    p[c0 + c + 1] = acc.y;
                }
            }
        }
        // recursive halving inside each group of eight lanes
#pragma unroll
        for (int o = 4, h = W / 2; o >= 1; o >>= 1, h >>= 1) {
            const bool hi = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < h; ++i) {
                const float send = hi ? p[i] : p[i + h];
                const float keep = hi ? p[i + h] : p[i];
                p[i] = keep + __shfl_xor_sync(KNNG_FULL_MASK, send, o);
            }
        }
        // lane (group g, g8) holds block 4c + g of points V * g8 + i
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float b0 = __shfl_sync(KNNG_FULL_MASK, p[i], g8);
            const float b1 = __shfl_sync(KNNG_FULL_MASK, p[i], 8 + g8);
            const float b2 = __shfl_sync(KNNG_FULL_MASK, p[i], 16 + g8);
            const float b3 = __shfl_sync(KNNG_FULL_MASK, p[i], 24 + g8);
            tot[i] = (((tot[i] + b0) + b1) + b2) + b3;
        }
    }
    // point c = lane % W is held as value c % V by the lanes with g8 = c / V
    const int c = lane % W;
    float out = 0.f;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const float v = __shfl_sync(KNNG_FULL_MASK, tot[i], c / V);
        if (c % V == i) out = v;
    }
    return out;
}

// Byte rows with exact integer distances (RowLoader::int_exact): the same
// lane split and reduction tree as warp_canon_dist_batch in 32-bit integer
// arithmetic, |x - y| per byte and a 4-way dot product per word.  Equal to
// the canonical FP32 distance, since every partial sum of that one is exact.
template <int W, int kDT>
__device__ __forceinline__ float warp_u8_dist_batch(const RowLoader<kDT>& L, int64_t a, const int* b, int nb)
{
    const int lane = threadIdx.x & 31;
    int bid[W];
#pragma unroll
    for (int c = 0; c < W; ++c) bid[c] = c < nb ? b[c] : (int)a;
    uint32_t p[W];
#pragma unroll
    for (int c = 0; c < W; ++c) p[c] = 0u;
    for (int j = 4 * lane; j < L.d; j += 128) {
        const uint32_t xa = L.load_u8x4(a, j);
        uint32_t xb[W];
#pragma unroll
        for (int c = 0; c < W; ++c) xb[c] = L.load_u8x4(bid[c], j);
#pragma unroll
        for (int c = 0; c < W; ++c) {
            const uint32_t t = __vabsdiffu4(xa, xb[c]);
            p[c] = __dp4a(t, t, p[c]);
        }
    }
#pragma unroll
    for (int o = 16; o >= W; o >>= 1) {
#pragma unroll
        for (int c = 0; c < W; ++c) p[c] += __shfl_xor_sync(KNNG_FULL_MASK, p[c], o);
    }
#pragma unroll
    for (int o = W / 2; o >= 1; o >>= 1) {
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const uint32_t send = hi ? p[i] : p[i + o];
            const uint32_t keep = hi ? p[i + o] : p[i];
            p[i] = keep + __shfl_xor_sync(KNNG_FULL_MASK, send, o);
        }
    }
    return (float)p[0];
}

// Canonical distances from a to b[0..nb) (nb <= 16): lane c < nb returns the
// distance to b[c].  Vector-aligned rows take the batched path; other rows
// one distance at a time.
template <int kDT>
__device__ __forceinline__ float warp_canon_dist16(const RowLoader<kDT>& L, int64_t a, const int* b, int nb)
{
    if (kDT == kDtU8 && L.all_vec() && L.int_exact()) return warp_u8_dist_batch<16>(L, a, b, nb);
    if (L.all_vec()) return warp_canon_dist_batch<16, kDT>(L, a, b, nb);
    const int lane = threadIdx.x & 31;
    float mine = 0.f;
    for (int c = 0; c < nb; ++c) {
        const float dd = warp_canon_dist(L, a, b[c]);
        if (lane == c) mine = dd;
    }
    return mine;
}

// Byte rows, 16-byte aligned with rows padded to a multiple of 16 bytes and
// d <= 128 (so every distance is an exact integer): eight lanes per
// candidate, lane l taking bytes 16 (l mod 8) .. + 15 of its row, so one load
// instruction fetches four whole rows.  load_query_u8 gives each lane its
// 16 bytes of the query row; score_u8_g8 writes the distances from a to
// b[0..nb) (nb <= 32) to out[0..nb) (shared memory).
__device__ __forceinline__ uint4 load_query_u8(const uint8_t* X, int64_t ld, int64_t a, int d)
{
    const int c = threadIdx.x & 7;
    const uint8_t* row = X + (uint64_t)(uint32_t)a * (uint32_t)ld;
    return 16 * c < d ? __ldg(reinterpret_cast<const uint4*>(row + 16 * c)) : make_uint4(0u, 0u, 0u, 0u);
}
__device__ __forceinline__ void score_u8_g8(const uint8_t* X, int64_t ld, int d, uint4 q, const int* b, int nb,
                                            float* out)
{
    const int lane = threadIdx.x & 31;
    const int c = lane & 7, g = lane >> 3;
    const bool has = 16 * c < d;
    uint4 x[8];
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int idx = 4 * it + g;
        x[it] = make_uint4(0u, 0u, 0u, 0u);
        if (idx < nb && has) {
            const uint8_t* row = X + (uint64_t)(uint32_t)b[idx] * (uint32_t)ld;
            x[it] = __ldg(reinterpret_cast<const uint4*>(row + 16 * c));
        }
    }
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        uint32_t t, acc = 0u;
        t = __vabsdiffu4(q.x, x[it].x); acc = __dp4a(t, t, acc);
        t = __vabsdiffu4(q.y, x[it].y); acc = __dp4a(t, t, acc);
        t = __vabsdiffu4(q.z, x[it].z); acc = __dp4a(t, t, acc);
        t = __vabsdiffu4(q.w, x[it].w); acc = __dp4a(t, t, acc);
        acc += __shfl_xor_sync(KNNG_FULL_MASK, acc, 4);
        acc += __shfl_xor_sync(KNNG_FULL_MASK, acc, 2);
        acc += __shfl_xor_sync(KNNG_FULL_MASK, acc, 1);
        const int idx = 4 * it + g;
        if (c == 0 && idx < nb) out[idx] = (float)acc;
    }
}

// Canonical distances from a to b[0..nb) (nb <= 32): lane c < nb returns the
// distance to b[c].  Byte rows with exact integer distances take one batch
// of 32 (32 rows in flight per warp), other rows two batches of 16.
template <int kDT>
__device__ __forceinline__ float warp_canon_dist32(const RowLoader<kDT>& L, int64_t a, const int* b, int nb)
{
    if (kDT == kDtU8 && L.all_vec() && L.int_exact()) return warp_u8_dist_batch<32>(L, a, b, nb);
    const int lane = threadIdx.x & 31;
    const float lo = warp_canon_dist16(L, a, b, min(nb, 16));
    float hi = 0.f;
    if (nb > 16) hi = warp_canon_dist16(L, a, b + 16, nb - 16);
    const float hi_l = __shfl_sync(KNNG_FULL_MASK, hi, lane & 15);
    return lane < 16 ? lo : hi_l;
}

// Rescoring of one row's candidate list (collective over one warp):
// keys[i * stride], i < nc <= 64, hold (D~, local index j); every candidate
// is rescored with the canonical FP32 distance between the original rows of
// lid[self] and lid[j], and the k best by (D, id) go to oi/od (padding -1 /
// +inf).  ws: kLeafWarpScratch bytes of the warp.
template <int kDT>
__device__ void leaf_rescore_list(const RowLoader<kDT>& L, const int32_t* lid, int self, const uint64_t* keys,
                                  int stride, int nc, int k, unsigned char* ws, int32_t* oi, float* od)
{
    const int lane = threadIdx.x & 31;
    int* cid = reinterpret_cast<int*>(ws);                   // 64 point ids
    uint64_t* rk = reinterpret_cast<uint64_t*>(ws + 1024);   // 64 rescored keys
    for (int c = lane; c < nc; c += 32) cid[c] = lid[(uint32_t)keys[(size_t)c * stride]];
    __syncwarp();
    const int gi = lid[self];
    for (int c0 = 0; c0 < nc; c0 += 16) {
        const int nb = min(16, nc - c0);
        const float dd = warp_canon_dist16(L, gi, cid + c0, nb);
        if (lane < nb) rk[c0 + lane] = pack_key(dd, (uint32_t)cid[c0 + lane]);
    }
    __syncwarp();
    uint64_t v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) v[e] = lane * 2 + e < nc ? rk[lane * 2 + e] : kKeyMax;
    warp_bitonic_sort<2>(v);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int i = lane * 2 + e;
        if (i < k) {
            const bool ok = i < nc;
            oi[i] = ok ? (int32_t)(uint32_t)v[e] : -1;
            od[i] = ok ? unord_key((uint32_t)(v[e] >> 32)) : __int_as_float(0x7f800000);
        }
    }
    __syncwarp();
}

// Finishes one row of a leaf graph (collective over one warp): from the
// candidate distances Drow(j), j in [0, m) local indices (j == self
// excluded), take the kp smallest (D~, j), rescore them with the canonical
// FP32 distance between the original rows, sort by (D, id) and write the k
// best to oi/od (padding with -1 / +inf).  lid maps local index -> point id
// (ascending with j, so a local index ranks like the id).
//
// With rescore == false the candidate distances are taken as final: the
// caller certifies that Drow(j) already equals the canonical distance (see
// the exactness test of the tensor-core path), and kp should be k.
//
// ws: per-warp shared scratch of kLeafWarpScratch bytes.  m <= 32 * PER.
constexpr int kLeafWarpScratch = 256 * 4 + 192 * 8;

// The kp (<= 64) best candidates of one row by (D~, local index), as local
// indices to out[0..min(kp, m - 1)) (collective over one warp; ws as
// above): the input of the staged FP32 rescoring.
template <int PER, class DFn>
__device__ void leaf_row_cands(const DFn& Drow, int m, int self, int kp, unsigned char* ws, uint16_t* out)
{
    const int lane = threadIdx.x & 31;
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws);
    uint64_t* keys = reinterpret_cast<uint64_t*>(ws + 1024);
    auto key = [&](int j) -> uint64_t { return j == self ? kKeyMax : pack_key(Drow(j), (uint32_t)j); };
    const int want = min(kp, m - 1);
    const int nsel = warp_topk_sorted<PER>(key, m, want, keys, keys + 64, hist);
    for (int c = lane; c < nsel; c += 32) out[c] = (uint16_t)(uint32_t)keys[c];
    __syncwarp();
}

template <int PER, int kDT, class DFn>
__device__ void leaf_row_finish(const RowLoader<kDT>& L, const DFn& Drow, int m, int self, const int32_t* lid,
                                int k, int kp, unsigned char* ws, int32_t* oi, float* od, bool rescore = true)
{
    const int lane = threadIdx.x & 31;
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws);
    uint64_t* keys = reinterpret_cast<uint64_t*>(ws + 1024);  // [0, 64) sorted picks, [64, 192) scratch
    auto key = [&](int j) -> uint64_t {
        return j == self ? kKeyMax : pack_key(Drow(j), (uint32_t)j);
    };
    const int want = min(kp, m - 1);
    if (want > 64) {
        // large k' (<= 128): radix select, then sort the picks
        const uint64_t thr = warp_select_threshold(key, m, want, hist);
        int* cand = reinterpret_cast<int*>(hist);  // the histogram is free again
        const int nsel = warp_compact_le(key, m, thr, cand);
        __syncwarp();
        const int gi = lid[self];
        uint64_t* rk = keys;  // 128 keys
        for (int c0 = 0; c0 < nsel; c0 += 16) {
            const int nb = min(16, nsel - c0);
            int* ids16 = reinterpret_cast<int*>(keys + 128);  // 16 point ids
            if (lane < nb) ids16[lane] = lid[cand[c0 + lane]];
            __syncwarp();
            float dd = 0.f;
            if (rescore) dd = warp_canon_dist16(L, gi, ids16, nb);
            else if (lane < nb) dd = Drow(cand[c0 + lane]);
            if (lane < nb) rk[c0 + lane] = pack_key(dd, (uint32_t)ids16[lane]);
            __syncwarp();
        }
        uint64_t v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = lane * 4 + e < nsel ? rk[lane * 4 + e] : kKeyMax;
        warp_bitonic_sort<4>(v);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = lane * 4 + e;
            if (i < k) {
                const bool ok = i < nsel;
                oi[i] = ok ? (int32_t)(uint32_t)v[e] : -1;
                od[i] = ok ? unord_key((uint32_t)(v[e] >> 32)) : __int_as_float(0x7f800000);
            }
        }
        __syncwarp();
        return;
    }
    const int nsel = warp_topk_sorted<PER>(key, m, want, keys, keys + 64, hist);
    uint64_t v[2];
    if (!rescore) {
        // picks are final: (distance, local index) -> (distance, point id)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int i = lane * 2 + e;
            v[e] = i < nsel ? ((keys[i] & 0xFFFFFFFF00000000ull) | (uint32_t)lid[(uint32_t)keys[i]]) : kKeyMax;
        }
    } else {
        int* cid = reinterpret_cast<int*>(hist);  // 64 point ids
        for (int c = lane; c < nsel; c += 32) cid[c] = lid[(uint32_t)keys[c]];
        __syncwarp();
        const int gi = lid[self];
        uint64_t* rk = keys + 64;
        for (int c0 = 0; c0 < nsel; c0 += 16) {
            const int nb = min(16, nsel - c0);
            const float dd = warp_canon_dist16(L, gi, cid + c0, nb);
            if (lane < nb) rk[c0 + lane] = pack_key(dd, (uint32_t)cid[c0 + lane]);
        }
        __syncwarp();
#pragma unroll
        for (int e = 0; e < 2; ++e) v[e] = lane * 2 + e < nsel ? rk[lane * 2 + e] : kKeyMax;
        warp_bitonic_sort<2>(v);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int i = lane * 2 + e;
        if (i < k) {
            const bool ok = i < nsel;
            oi[i] = ok ? (int32_t)(uint32_t)v[e] : -1;
            od[i] = ok ? unord_key((uint32_t)(v[e] >> 32)) : __int_as_float(0x7f800000);
        }
    }
    __syncwarp();
}

}  // namespace knng

