// Random divisions (Sec. 3.1 of arXiv:1307.7852; split rule of the appendix
// after Lemma 1): every tree recursively bisects its nodes at the median of
// the projections onto a Philox random direction, until a node holds at most
// g points.
//
// GPU form: all T trees advance together, one level per step.
//   1. gen_dirs   -- the directions of the level's split nodes, from Philox.
//   2. project    -- one warp per point reads the point's row ONCE and
//                    projects it on the direction of its node in every tree
//                    (fixed-order FP32, bit-identical to the CPU definition);
//                    the 32-bit key lands at the point's current position.
//   3. select     -- per node, the floor(m/2)-th smallest 64-bit key
//                    (ord(s) << 32 | id) by radix select: one block per node
//                    for nodes <= kSmallCap, otherwise block-private
//                    histograms merged in global memory, one digit per pass.
//   4. scatter    -- stable partition of each node into its two children.
// Stability makes every node's segment ascend by id, so the leaves come out
// in canonical order without a final sort.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include <type_traits>

#include "knng_common.cuh"
#include "knng_internal.h"
#include "tc_ptx.cuh"

namespace knng {

// ---------------------------------------------------------------------------
// Host: the tree shape.  Sizes at a level are floor/ceil halves, so the
// shape depends on (n, g) only and is shared by all trees.
// ---------------------------------------------------------------------------
void make_forest_plan(const std::vector<int64_t>& roots, int g, TreePlan& P)
{
    int64_t n = 0;
    for (int64_t r : roots) n += r;
    P.n = n;
    P.g = g;
    P.roots = roots;
    P.levels.clear();
    P.nodes.clear();
    P.chunks.clear();
    P.leaf_off.clear();
    P.max_nodes = 0;
    P.max_chunks = 0;
    P.max_big_nodes = 0;
    P.max_leaf = 0;

    struct Tmp {
        uint32_t v;
        int64_t off, size;
        int parent;  // index in the previous level's (sorted) list
        int side;    // 0 left, 1 right
    };
    std::vector<Tmp> cur;
    std::vector<std::pair<int64_t, int64_t>> leaves;  // (off, size)
    int64_t off = 0;
    for (int64_t r : roots) {
        if (r > g) cur.push_back({0u, off, r, -1, 0});
        else if (r > 0) leaves.push_back({off, r});
        off += r;
    }
    while (!cur.empty()) {
        // big nodes first, then small ones, each group in offset order
        std::stable_sort(cur.begin(), cur.end(), [](const Tmp& a, const Tmp& b) {
            return (a.size > kSmallCap) > (b.size > kSmallCap);
        });
        // link the parents of the previous level to these positions
        if (!P.levels.empty()) {
            const LevelPlan& prev = P.levels.back();
            for (size_t i = 0; i < cur.size(); ++i) {
                SplitNode& pn = P.nodes[prev.node_base + cur[i].parent];
                if (cur[i].side == 0) pn.childL = (int32_t)i;
                else pn.childR = (int32_t)i;
            }
        }
        LevelPlan L;
        L.node_base = (int64_t)P.nodes.size();
        L.nnodes = (int32_t)cur.size();
        L.nbig = 0;
        L.max_small = 0;
        std::vector<Tmp> nxt;
        for (size_t i = 0; i < cur.size(); ++i) {
            const Tmp& t = cur[i];
            SplitNode s{};
            s.v = t.v;
            s.off = (int32_t)t.off;
            s.size = (int32_t)t.size;
            s.childL = -1;
            s.childR = -1;
            const int64_t ml = t.size / 2, mr = t.size - ml;
            if (ml > g) nxt.push_back({2 * t.v, t.off, ml, (int)i, 0});
            else leaves.push_back({t.off, ml});
            if (mr > g) nxt.push_back({2 * t.v + 1, t.off + ml, mr, (int)i, 1});
            else leaves.push_back({t.off + ml, mr});
            P.nodes.push_back(s);
            if (t.size > kSmallCap) ++L.nbig;
            else L.max_small = std::max<int32_t>(L.max_small, (int32_t)t.size);
        }
        L.chunk_base = (int64_t)P.chunks.size();
        L.nchunks = 0;
        for (int32_t s = 0; s < L.nbig; ++s) {
            const SplitNode& sn = P.nodes[L.node_base + s];
            const int32_t first = L.nchunks;
            for (int64_t a = 0; a < sn.size; a += kChunk) {
                Chunk c;
                c.node = s;
                c.start = (int32_t)(sn.off + a);
                c.len = (int32_t)std::min<int64_t>(kChunk, sn.size - a);
                c.first = first;
                P.chunks.push_back(c);
                ++L.nchunks;
            }
        }
        P.max_nodes = std::max(P.max_nodes, L.nnodes);
        P.max_big_nodes = std::max(P.max_big_nodes, L.nbig);
        P.max_chunks = std::max(P.max_chunks, L.nchunks);
        P.levels.push_back(L);
        cur.swap(nxt);
    }
    std::sort(leaves.begin(), leaves.end());
    for (auto& l : leaves) {
        P.leaf_off.push_back((int32_t)l.first);
        P.max_leaf = std::max<int32_t>(P.max_leaf, (int32_t)l.second);
    }
    P.leaf_off.push_back((int32_t)n);
}

void make_tree_plan(int64_t n, int g, TreePlan& P)
{
    make_forest_plan(std::vector<int64_t>{n}, g, P);
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
__global__ void init_perm_kernel(int64_t n, int T, int first_node, int32_t* perm, int32_t* pos_of,
                                 int32_t* node_of, int32_t* node_pos)
{
    const int64_t total = (int64_t)T * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(e % n);
        perm[e] = i;
        pos_of[e] = i;
        node_of[e] = first_node;
        node_pos[e] = first_node;
    }
}

// Points of the root node s of level 0 start in node s (other points are in
// roots that are already leaves and keep node -1).  At level 0 positions are
// ids, so the map by id and the map by position start equal.
// Block (x, s, t): slice x of root s in tree t.
__global__ void init_root_nodes_kernel(int64_t n, const SplitNode* __restrict__ nodes, int32_t* node_of,
                                       int32_t* node_pos)
{
    const SplitNode nd = nodes[blockIdx.y];
    int32_t* row = node_of + (int64_t)blockIdx.z * n;
    int32_t* prow = node_pos + (int64_t)blockIdx.z * n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nd.size; e += gridDim.x * blockDim.x) {
        row[nd.off + e] = (int32_t)blockIdx.y;
        prow[nd.off + e] = (int32_t)blockIdx.y;
    }
}

// dirs[t][s][0..d_pad): direction of split node s of this level in tree
// t0 + t (a tree's directions depend on its own index only).
__global__ void gen_dirs_kernel(float* dirs, int T, int S, int d, int d_pad,
                                const SplitNode* nodes, uint32_t level, uint64_t seed, uint32_t t0)
{
    const int q4 = d_pad / 4;
    const int64_t total = (int64_t)T * S * q4;
    const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e % q4);
        const int s = (int)((e / q4) % S);
        const int t = (int)(e / ((int64_t)q4 * S));
        const uint4 w = philox4x32_10(make_uint4(t0 + (uint32_t)t, level, nodes[s].v, (uint32_t)q), key);
        const int j = 4 * q;
        float4 a;
        a.x = (j + 0 < d) ? tri_entry(w.x) : 0.f;
        a.y = (j + 1 < d) ? tri_entry(w.y) : 0.f;
        a.z = (j + 2 < d) ? tri_entry(w.z) : 0.f;
        a.w = (j + 3 < d) ? tri_entry(w.w) : 0.f;
        reinterpret_cast<float4*>(dirs)[e] = a;
    }
}

// Learned splits, step 1: range (as order keys) of every tree's feature of
// this level inside every node.  Positions are visited in node order, so the
// lanes of a warp nearly always share one node: the warp then reduces its
// keys and one lane updates the node's range (on the top levels every point
// of a tree would otherwise hit the same two words).
struct FeatOfTree {
    int f[32];
};
__global__ void node_feature_range_kernel(int64_t n, int T, const float* __restrict__ Z, int C, FeatOfTree ft,
                                          const int32_t* __restrict__ node_pos, const int32_t* __restrict__ perm,
                                          int S, uint32_t* __restrict__ rmin, uint32_t* __restrict__ rmax)
{
    const int64_t total = (int64_t)T * n;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x; e0 < total; e0 += stride) {
        const int64_t e = e0 + threadIdx.x;
        int64_t key = -1;  // (tree, node), -1: nothing to add
        uint32_t o = 0;
        if (e < total) {
            const int sn = node_pos[e];
            if (sn >= 0) {
                const int t = (int)(e / n);
                key = (int64_t)t * S + sn;
                o = ord_key(Z[(int64_t)perm[e] * C + ft.f[t]]);
            }
        }
        const int64_t key0 = __shfl_sync(KNNG_FULL_MASK, key, 0);
        if (__all_sync(KNNG_FULL_MASK, key == key0)) {
            if (key0 < 0) continue;
            const uint32_t mn = __reduce_min_sync(KNNG_FULL_MASK, o);
            const uint32_t mx = __reduce_max_sync(KNNG_FULL_MASK, o);
            if (lane == 0) {
                atomicMin(&rmin[key0], mn);
                atomicMax(&rmax[key0], mx);
            }
        } else if (key >= 0) {
            atomicMin(&rmin[key], o);
            atomicMax(&rmax[key], o);
        }
    }
}

// Range of every feature over all points (order keys in scratch, then
// max - min in frange).  C divides 32 and every thread's stride, so a thread
// only ever sees feature gtid mod C: it keeps its own minimum and maximum,
// the lanes of a warp holding the same feature combine theirs, and one
// atomic per warp and feature remains (not one per element).
__global__ void feature_range_kernel(const float* __restrict__ Z, int64_t n, int C, uint32_t* __restrict__ mm)
{
    const int lane = threadIdx.x & 31;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t mn = 0xFFFFFFFFu, mx = 0u;
    for (int64_t e = gtid; e < n * C; e += stride) {
        const uint32_t o = ord_key(Z[e]);
        mn = min(mn, o);
        mx = max(mx, o);
    }
    for (int o = 16; o >= C; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(KNNG_FULL_MASK, mn, o));
        mx = max(mx, __shfl_xor_sync(KNNG_FULL_MASK, mx, o));
    }
    if (lane < C) {
        atomicMin(&mm[lane], mn);
        atomicMax(&mm[C + lane], mx);
    }
}
__global__ void feature_range_finish_kernel(int C, const uint32_t* __restrict__ mm, float* __restrict__ frange)
{
    const int c = threadIdx.x;
    if (c < C) frange[c] = unord_key(mm[C + c]) - unord_key(mm[c]);
}

cudaError_t run_feature_range(const float* Z, int64_t n, int C, uint32_t* mm, float* frange, cudaStream_t st)
{
    if (C < 1 || C > 32 || (32 % C) != 0) return cudaErrorInvalidValue;
    cudaMemsetAsync(mm, 0xFF, sizeof(uint32_t) * C, st);
    cudaMemsetAsync(mm + C, 0, sizeof(uint32_t) * C, st);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n * C + 255) / 256, (int64_t)num_sms() * 8));
    feature_range_kernel<<<blocks, 256, 0, st>>>(Z, n, C, mm);
    feature_range_finish_kernel<<<1, 32, 0, st>>>(C, mm, frange);
    note_launches(2);
    return cudaGetLastError();
}

// Learned-split settings of one level, passed to the projection kernel.
struct LevelFeat {
    const float* Z;
    int C;
    FeatOfTree ft;
    const uint32_t* rmin;
    const uint32_t* rmax;
    const float* frange;
    float tau;
};

void learned_feature_order(uint64_t seed, int T, int C, LearnedFeat& lf)
{
    const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    for (int t = 0; t < T && t < 32; ++t) {
        for (int c = 0; c < C; ++c) lf.feat[t][c] = c;
        for (int i = C - 1; i > 0; --i) {
            const uint4 w = philox4x32_10(make_uint4((uint32_t)t, 0x4C524E44u, (uint32_t)i, 0u), key);
            const int j = (int)(w.x % (uint32_t)(i + 1));
            const int tmp = lf.feat[t][i];
            lf.feat[t][i] = lf.feat[t][j];
            lf.feat[t][j] = tmp;
        }
    }
}

// One warp per point; up to 8 trees per pass over the row.  The projection
// order is the canonical one: lane l, j = 128c + 4l + e, fmaf, then the
// pairwise rounds 16..1.
template <bool kLearned, class Loader>
__device__ __forceinline__ void project_body(const Loader& L, int64_t n, int T, const float* __restrict__ dirs,
                                             int S, int d_pad, const int32_t* __restrict__ node_of,
                                             const int32_t* __restrict__ pos_of, uint32_t* __restrict__ keys,
                                             const LevelFeat& lv)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        // the warp's next row streams into L2 while this one is projected: the
        // chunk loads below then wait on L2, not on DRAM
        if (i + nwarps < n) L.prefetch_l2(i + nwarps, lane);
        for (int t0 = 0; t0 < T; t0 += 8) {
            const int tl = t0 + lane;
            const int my_s = (lane < 8 && tl < T) ? node_of[(int64_t)tl * n + i] : -1;
            if (__ballot_sync(KNNG_FULL_MASK, my_s >= 0) == 0) continue;
            // learned levels: a node splits on its learned feature while the
            // feature still varies there, and then needs no projection
            bool my_feat = false;
            if (kLearned && my_s >= 0) {
                const int f = lv.ft.f[tl];
                const int64_t ns = (int64_t)tl * S + my_s;
                const float span = unord_key(lv.rmax[ns]) - unord_key(lv.rmin[ns]);
                my_feat = span > lv.tau * lv.frange[f];
            }
            const int proj_s = my_feat ? -1 : my_s;
            int sv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) sv[u] = __shfl_sync(KNNG_FULL_MASK, proj_s, u);
            if (kLearned && __ballot_sync(KNNG_FULL_MASK, proj_s >= 0) == 0) {
                if (my_s >= 0) {
                    const int64_t row = (int64_t)tl * n;
                    keys[row + pos_of[row + i]] = ord_key(lv.Z[i * lv.C + lv.ft.f[tl]]);
                }
                continue;
            }
            float acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = 0.0f;
            for (int j = 4 * lane; j < L.d; j += 128) {
                const float4 x = L.load4(i, j);
                const bool full = j + 3 < L.d;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (sv[u] < 0) continue;
                    const float4 a = *reinterpret_cast<const float4*>(
                        dirs + ((int64_t)(t0 + u) * S + sv[u]) * d_pad + j);
                    if (full) {
                        acc[u] = fmaf(x.x, a.x, acc[u]);
                        acc[u] = fmaf(x.y, a.y, acc[u]);
                        acc[u] = fmaf(x.z, a.z, acc[u]);
                        acc[u] = fmaf(x.w, a.w, acc[u]);
                    } else {
                        acc[u] = fmaf(x.x, a.x, acc[u]);
                        if (j + 1 < L.d) acc[u] = fmaf(x.y, a.y, acc[u]);
                        if (j + 2 < L.d) acc[u] = fmaf(x.z, a.z, acc[u]);
                    }
                }
            }
            float mine = 0.0f;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) acc[u] += __shfl_xor_sync(KNNG_FULL_MASK, acc[u], o);
                if (lane == u) mine = acc[u];
            }
            if (my_s >= 0) {
                const int64_t row = (int64_t)tl * n;
                const uint32_t key = my_feat ? ord_key(lv.Z[i * lv.C + lv.ft.f[tl]]) : ord_key(mine);
                keys[row + pos_of[row + i]] = key;
            }
        }
    }
}

// Float rows whose byte copy is exact (*xb_bad == 0, see XDesc) are read from
// the copy: the same float values, a quarter of the bytes.  With
// bytes_elsewhere set, such a build is left to project_bytes_kernel.
template <int kDT, bool kLearned>
__global__ void __launch_bounds__(256) project_kernel(RowLoader<kDT> L, RowLoader<kDtU8> Lb,
                                                      const int* __restrict__ xb_bad, bool bytes_elsewhere,
                                                      int64_t n, int T, const float* __restrict__ dirs, int S,
                                                      int d_pad, const int32_t* __restrict__ node_of,
                                                      const int32_t* __restrict__ pos_of,
                                                      uint32_t* __restrict__ keys, LevelFeat lv)
{
    if constexpr (kDT == kDtF32) {
        if (xb_bad && *xb_bad == 0) {
            if (bytes_elsewhere) return;
            project_body<kLearned>(Lb, n, T, dirs, S, d_pad, node_of, pos_of, keys, lv);
            return;
        }
    }
    project_body<kLearned>(L, n, T, dirs, S, d_pad, node_of, pos_of, keys, lv);
}

// Exact floats of the four bytes of w: the byte permute assembles 2^23 + b
// (the exponent of 2^23 with b in the low mantissa bits) and one packed add
// takes 2^23 off two of them at a time; both steps are exact.  This keeps
// the conversion off the integer-to-float unit, which runs at a quarter of
// the FMA rate.
__device__ __forceinline__ void bytes_exact4(uint32_t w, float& x0, float& x1, float& x2, float& x3)
{
    const float2 off = make_float2(-8388608.0f, -8388608.0f);
    const float2 lo = __fadd2_rn(make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u)),
                                             __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7541u))),
                                 off);
    const float2 hi = __fadd2_rn(make_float2(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7542u)),
                                             __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7543u))),
                                 off);
    x0 = lo.x;
    x1 = lo.y;
    x2 = hi.x;
    x3 = hi.y;
}

// Lane partial of the canonical order over one 4-byte word: s plus
// x[j..j+3] . a[j..j+3] by four fmaf in j order.
__device__ __forceinline__ float word_partial(uint32_t w, const float4& a, float s)
{
    float x0, x1, x2, x3;
    bytes_exact4(w, x0, x1, x2, x3);
    s = fmaf(x0, a.x, s);
    s = fmaf(x1, a.y, s);
    s = fmaf(x2, a.z, s);
    return fmaf(x3, a.w, s);
}

// Rows of at most 128 bytes (one canonical chunk): the value of lane
// partial L after the pairwise rounds down to distance O (O = 32: the
// partial itself), evaluated depth-first so that few sums are live at once.
// Partial L covers bytes 4L .. 4L + 3; words past the row (L >= nw) and
// direction entries past d contribute nothing (the row's padding bytes and
// the direction's padding entries are zeros, and adding +0 * 0 to a partial,
// which is never -0, leaves it unchanged).
template <int L, int O, bool kFull>
struct ProjTree {
    static __device__ __forceinline__ float eval(const uint32_t (&w)[32], const float* __restrict__ a, int nw,
                                                 int d)
    {
        return ProjTree<L, 2 * O, kFull>::eval(w, a, nw, d) + ProjTree<L + O, 2 * O, kFull>::eval(w, a, nw, d);
    }
};
template <int L, bool kFull>
struct ProjTree<L, 32, kFull> {
    static __device__ __forceinline__ float eval(const uint32_t (&w)[32], const float* __restrict__ a, int nw,
                                                 int d)
    {
        if (kFull) return word_partial(w[L], __ldg(reinterpret_cast<const float4*>(a + 4 * L)), 0.0f);
        if (L >= nw || 4 * L >= d) return 0.0f;
        return word_partial(w[L], __ldg(reinterpret_cast<const float4*>(a + 4 * L)), 0.0f);
    }
};

// Node-major projection of byte rows (16-byte aligned, rows padded to
// multiples of 16 bytes with zeros, or byte input of such rows): one thread
// per (tree, position), a warp on 32 consecutive positions, which mostly
// share their node, so a direction load is one broadcast.  The thread forms
// the 32 lane partials of the canonical order (lane l: j = 128c + 4l + e,
// fmaf) and the pairwise rounds 16, 8, 4, 2, 1 itself, so the value is the
// one of the warp-cooperative projection bit for bit.  Rows of at most 128
// bytes (kOneChunk) are fetched by the warp eight lanes to a row (one
// 128-byte line per four lanes' loads instead of one line per lane and
// load) into shared memory, and each thread then sums its row depth-first;
// longer rows are gathered by their threads.  The node comes from the map
// by position.  Unless bytes_given, it runs only when the byte copy of
// float rows is exact (*xb_bad == 0).
template <bool kOneChunk, bool kFull>
__global__ void __launch_bounds__(256, 4) project_bytes_kernel(RowLoader<kDtU8> Lb, const int* __restrict__ xb_bad,
                                                               bool bytes_given, int64_t n, int T,
                                                               const float* __restrict__ dirs, int S, int d_pad,
                                                               const int32_t* __restrict__ cur,
                                                               const int32_t* __restrict__ node_pos,
                                                               uint32_t* __restrict__ keys)
{
    // rows staged per warp: 32 rows of 8 16-byte words, stride 9 words (the
    // 16-byte accesses of eight lanes fall in distinct banks)
    __shared__ uint4 srow[8][32][9];
    if (!bytes_given && (!xb_bad || *xb_bad != 0)) return;
    const int d = Lb.d;
    const int nq = (d + 15) >> 4;  // 16-byte words of a row
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int64_t total = (int64_t)T * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // a multiple of 32
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int t = (int)(g / n);
    int64_t i = g - (int64_t)t * n;  // position within tree t (g = t n + i)
    const uint8_t* X = static_cast<const uint8_t*>(Lb.X);
    for (; g - lane < total; g += stride) {  // whole warps iterate together
        const bool valid = g < total;
        const int tt = t;
        i += stride;
        while (i >= n && t < T) {
            i -= n;
            ++t;
        }
        const int32_t id = valid ? cur[g] : 0;
        const int sn = valid ? node_pos[g] : -1;  // -1: a leaf of an earlier level
        float v = 0.f;
        if constexpr (kOneChunk) {
            // the warp's rows, eight lanes to a row
            const int q = lane & 7;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int rr = 4 * r + (lane >> 3);
                const int32_t idr = __shfl_sync(KNNG_FULL_MASK, id, rr);
                const int snr = __shfl_sync(KNNG_FULL_MASK, sn, rr);
                uint4 u = make_uint4(0u, 0u, 0u, 0u);
                if (snr >= 0 && (kFull || q < nq))
                    u = __ldg(reinterpret_cast<const uint4*>(X + Lb.row_off(idr) + 16 * q));
                srow[wq][rr][q] = u;
            }
            __syncwarp();
            if (sn >= 0) {
                uint32_t w[32];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const uint4 u = srow[wq][lane][c];
                    w[4 * c + 0] = u.x;
                    w[4 * c + 1] = u.y;
                    w[4 * c + 2] = u.z;
                    w[4 * c + 3] = u.w;
                }
                const float* a = dirs + ((int64_t)tt * S + sn) * d_pad;
                v = ProjTree<0, 1, kFull>::eval(w, a, 4 * nq, d);
            }
            __syncwarp();  // the rows are read before the next batch lands
        } else {
            if (sn >= 0) {
                const uint8_t* row = X + Lb.row_off(id);
                const float* a = dirs + ((int64_t)tt * S + sn) * d_pad;
                float acc[32];
#pragma unroll
                for (int l = 0; l < 32; ++l) acc[l] = 0.f;
                for (int c0 = 0; c0 < d; c0 += 128) {
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        const int jb = c0 + 16 * qq;  // bytes jb .. jb + 15: lanes 4qq .. 4qq + 3
                        if (jb < d) {
                            const uint4 u = __ldg(reinterpret_cast<const uint4*>(row + jb));
                            const uint32_t wv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const int j = jb + 4 * h;
                                if (j < d)
                                    acc[4 * qq + h] = word_partial(
                                        wv[h], __ldg(reinterpret_cast<const float4*>(a + j)), acc[4 * qq + h]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1)
#pragma unroll
                    for (int l = 0; l < o; ++l) acc[l] = acc[l] + acc[l + o];
                v = acc[0];
            }
        }
        if (sn >= 0) keys[g] = ord_key(v);
    }
}

// The same projection with the rows fetched by the tensor memory
// accelerator (rows of at most 128 bytes): per warp, one lane gathers the
// batch's 32 rows, four per gather4 copy, as 144-byte rows (bytes past the
// tensor's rows read as zeros) into 128-byte aligned groups of four, and the
// copies complete on the warp's mbarrier.  The waits are bounded: a warp
// that gives up sets the error word, waits once more for its copies and
// leaves.
constexpr int kTmaRow = 144;    // bytes per gathered row
constexpr int kTmaGroup = 640;  // bytes per group of four rows (128-byte aligned)
constexpr long long kProjWait = 2000000000LL;  // ~1 s at GB300 clocks
template <bool kFull>
__global__ void __launch_bounds__(256, 4) project_bytes_tma_kernel(const __grid_constant__ CUtensorMap tmap, int d,
                                                                   const int* __restrict__ xb_bad, bool bytes_given,
                                                                   int64_t n, int T, const float* __restrict__ dirs,
                                                                   int S, int d_pad, const int32_t* __restrict__ cur,
                                                                   const int32_t* __restrict__ node_pos,
                                                                   uint32_t* __restrict__ keys, int* err)
{
    __shared__ __align__(128) unsigned char srow[8][8 * kTmaGroup];
    __shared__ int sid[8][32];
    __shared__ __align__(8) uint64_t bar[8];
    if (!bytes_given && (!xb_bad || *xb_bad != 0)) return;
    const int nq = (d + 15) >> 4;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    unsigned char* buf = srow[wq];
    if (lane == 0) {
        tc::mbar_init(&bar[wq], 1);
        tc::fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    const int64_t total = (int64_t)T * n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;  // a multiple of 32
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int t = (int)(g / n);
    int64_t i = g - (int64_t)t * n;  // position within tree t (g = t n + i)
    for (; g - lane < total; g += stride) {  // whole warps iterate together
        const bool valid = g < total;
        const int tt = t;
        i += stride;
        while (i >= n && t < T) {
            i -= n;
            ++t;
        }
        const int32_t id = valid ? cur[g] : 0;
        const int sn = valid ? node_pos[g] : -1;  // -1: a leaf of an earlier level
        sid[wq][lane] = sn >= 0 ? id : 0;          // any row for a position without work
        // the previous batch's rows are read (generic proxy) before the
        // copies (async proxy) overwrite them
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
            tc::mbar_arrive_expect_tx(&bar[wq], 32 * kTmaRow);
#pragma unroll
            for (int r = 0; r < 8; ++r)
                tc::tma_gather4_2d(buf + r * kTmaGroup, &tmap, &bar[wq], 0, sid[wq][4 * r], sid[wq][4 * r + 1],
                                   sid[wq][4 * r + 2], sid[wq][4 * r + 3]);
        }
        const bool ok = __all_sync(KNNG_FULL_MASK, tc::mbar_wait(&bar[wq], phase, kProjWait));
        if (!ok) {
            if (lane == 0) {
                if (err) atomicExch(err, 1);
                tc::mbar_wait(&bar[wq], phase, kProjWait);
            }
            __syncwarp();
            return;
        }
        phase ^= 1u;
        if (sn >= 0) {
            // the rows of two groups share their banks (groups are 128-byte
            // aligned): lanes of odd groups read their 16-byte words in the
            // order c ^ 4, so the eight lanes of a phase hit 32 distinct banks
            uint32_t w[32];
            const uint4* rowp = reinterpret_cast<const uint4*>(buf + (lane >> 2) * kTmaGroup + (lane & 3) * kTmaRow);
            const bool odd = (lane & 4) != 0;
            uint4 v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = rowp[odd ? (c ^ 4) : c];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const uint4 u = odd ? v[c ^ 4] : v[c];
                w[4 * c + 0] = u.x;
                w[4 * c + 1] = u.y;
                w[4 * c + 2] = u.z;
                w[4 * c + 3] = u.w;
            }
            const float* a = dirs + ((int64_t)tt * S + sn) * d_pad;
            keys[g] = ord_key(ProjTree<0, 1, kFull>::eval(w, a, 4 * nq, d));
        }
    }
}

// ---- block radix select (one block, keys in shared memory) ---------------
template <int NT>
__device__ unsigned long long block_select(const unsigned long long* k64, int m, int want,
                                           uint32_t* hist, uint32_t* bcast)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    unsigned long long prefix = 0, mask = 0;
    int rank = want;
    for (int shift = 56;; shift -= 8) {
        for (int b = tid; b < 256; b += NT) hist[b] = 0;
        __syncthreads();
        for (int e = tid; e < m; e += NT) {
            const unsigned long long kv = k64[e];
            if ((kv & mask) == prefix) atomicAdd(&hist[(kv >> shift) & 0xFF], 1u);
        }
        __syncthreads();
        if (w == 0) {
            uint32_t c[8], lsum = 0;
#pragma unroll
            for (int b = 0; b < 8; ++b) { c[b] = hist[lane * 8 + b]; lsum += c[b]; }
            uint32_t incl = lsum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(KNNG_FULL_MASK, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t excl = incl - lsum;
            if (excl < (uint32_t)rank && (uint32_t)rank <= incl) {
                uint32_t run = excl;
                bool found = false;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    if (!found && run < (uint32_t)rank && (uint32_t)rank <= run + c[b]) {
                        bcast[0] = lane * 8 + b;
                        bcast[1] = run;
                        bcast[2] = c[b];
                        found = true;
                    }
                    run += c[b];
                }
            }
        }
        __syncthreads();
        const uint32_t digit = bcast[0], before = bcast[1], inbin = bcast[2];
        prefix |= (unsigned long long)digit << shift;
        mask |= 0xFFull << shift;
        rank -= (int)before;
        __syncthreads();
        if ((uint32_t)rank == inbin || shift == 0)
            return prefix | (shift ? ((1ull << shift) - 1) : 0ull);
    }
}

// Exclusive block scan of one int per thread; returns the prefix, and the
// total in *total.
template <int NT>
__device__ int block_excl_scan(int v, int* sh, int* total)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(KNNG_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        int s = lane < NT / 32 ? sh[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(KNNG_FULL_MASK, si, o);
            if (lane >= o) si += t;
        }
        if (lane < NT / 32) sh[lane] = si - s;
        if (lane == NT / 32 - 1) sh[32] = si;
    }
    __syncthreads();
    const int r = sh[w] + incl - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// Stable two-way scatter of elements [0, len) of a slice (keys in shared
// memory) in rounds of NT consecutive elements: a block-wide count of the
// left elements before each one gives its destination, so a warp's left and
// right elements land in two contiguous runs.  lbase/rbase: destination of
// the slice's first left / right element.  The node of every destination
// position is written to node_pos; the maps by id (pos_of, node_of) only
// when a later projection reads them (id_maps).
template <int NT>
__device__ void stable_scatter(const unsigned long long* k64, int len, unsigned long long thr,
                               int32_t lbase, int32_t rbase, int32_t childL, int32_t childR,
                               int32_t* perm_nxt, int32_t* node_pos, int32_t* pos_of, int32_t* node_of,
                               bool id_maps, int* sh)
{
    constexpr int NW = NT / 32;
    static_assert(NW <= 16, "two rounds of warp counts share sh[0..31]");
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int before = 0;  // left elements of the earlier rounds
    for (int base = 0, r = 0; base < len; base += NT, r ^= 1) {
        const int e = base + tid;
        const unsigned long long kv = e < len ? k64[e] : ~0ull;
        const bool left = e < len && kv <= thr;
        const uint32_t b = __ballot_sync(KNNG_FULL_MASK, left);
        // the counts alternate between two halves of sh: one barrier a round
        if (lane == 0) sh[16 * r + w] = __popc(b);
        __syncthreads();
        int pre = 0, tot = 0;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            const int c = sh[16 * r + i];
            pre += i < w ? c : 0;
            tot += c;
        }
        if (e < len) {
            const int lrank = before + pre + __popc(b & lanemask_lt());
            const int32_t id = (int32_t)(uint32_t)kv;
            const int32_t dst = left ? lbase + lrank : rbase + (e - lrank);
            const int32_t child = left ? childL : childR;
            perm_nxt[dst] = id;
            node_pos[dst] = child;
            if (id_maps) {
                pos_of[id] = dst;
                node_of[id] = child;
            }
        }
        before += tot;
    }
}

// Whether this level's scatter keeps the maps by id: 1 always, 0 never,
// 2 when the float rows' byte copy is not exact (*xb_bad != 0: the next
// level then projects by id).
__device__ __forceinline__ bool want_id_maps(int id_mode, const int* xb_bad)
{
    return id_mode == 1 || (id_mode == 2 && xb_bad && *xb_bad != 0);
}

// One block per (split node, tree), node <= kSmallCap points.
template <int NT>
__global__ void __launch_bounds__(NT) split_small_kernel(int64_t n, const SplitNode* __restrict__ nodes,
                                                         const uint32_t* __restrict__ keys,
                                                         const int32_t* __restrict__ perm_cur,
                                                         int32_t* perm_nxt, int32_t* node_pos, int32_t* pos_of,
                                                         int32_t* node_of, int id_mode, const int* xb_bad)
{
    extern __shared__ unsigned long long k64[];
    __shared__ uint32_t hist[256];
    __shared__ uint32_t bcast[4];
    __shared__ int sh[33];
    const SplitNode nd = nodes[blockIdx.x];
    const int64_t row = (int64_t)blockIdx.y * n;
    const int m = nd.size;
    for (int e = threadIdx.x; e < m; e += NT)
        k64[e] = ((unsigned long long)keys[row + nd.off + e] << 32) | (uint32_t)perm_cur[row + nd.off + e];
    __syncthreads();
    const unsigned long long thr = block_select<NT>(k64, m, m / 2, hist, bcast);
    stable_scatter<NT>(k64, m, thr, nd.off, nd.off + m / 2, nd.childL, nd.childR, perm_nxt + row,
                       node_pos + row, pos_of + row, node_of + row, want_id_maps(id_mode, xb_bad), sh);
}

// ---- multi-block split of large nodes ------------------------------------
__global__ void big_init_kernel(int S, int T, const SplitNode* nodes, SelState* st)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S * T) return;
    SelState s;
    s.prefix = 0;
    s.mask = 0;
    s.thr = 0;
    s.rank = nodes[e % S].size / 2;
    s.done = 0;
    st[e] = s;
}

template <int NT>
__global__ void __launch_bounds__(NT) big_hist_kernel(int64_t n, int shift, int S, const Chunk* __restrict__ chunks,
                                                      const uint32_t* __restrict__ keys,
                                                      const int32_t* __restrict__ perm,
                                                      const SelState* __restrict__ st, uint32_t* ghist)
{
    __shared__ uint32_t h[256];
    const Chunk c = chunks[blockIdx.x];
    const int t = blockIdx.y;
    const SelState s = st[(int64_t)t * S + c.node];
    if (s.done) return;
    for (int b = threadIdx.x; b < 256; b += NT) h[b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)t * n + c.start;
    for (int e = threadIdx.x; e < c.len; e += NT) {
        const unsigned long long kv = ((unsigned long long)keys[base + e] << 32) | (uint32_t)perm[base + e];
        if ((kv & s.mask) == s.prefix) atomicAdd(&h[(kv >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    uint32_t* g = ghist + ((int64_t)t * S + c.node) * 256;
    for (int b = threadIdx.x; b < 256; b += NT)
        if (h[b]) atomicAdd(&g[b], h[b]);
}

// One warp per (node, tree): choose the digit of this pass.
__global__ void big_pick_kernel(int shift, int S, SelState* st, uint32_t* ghist)
{
    const int lane = threadIdx.x;
    const int64_t e = (int64_t)blockIdx.y * S + blockIdx.x;
    SelState s = st[e];
    if (s.done) return;
    uint32_t* h = ghist + e * 256;
    uint32_t c[8], lsum = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) { c[b] = h[lane * 8 + b]; lsum += c[b]; h[lane * 8 + b] = 0; }
    uint32_t incl = lsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(KNNG_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t excl = incl - lsum;
    const uint32_t rank = (uint32_t)s.rank;
    const bool mine = excl < rank && rank <= incl;
    const uint32_t owner = __ffs(__ballot_sync(KNNG_FULL_MASK, mine)) - 1;
    uint32_t digit = 0, before = 0, inbin = 0;
    if (mine) {
        uint32_t run = excl;
        bool found = false;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            if (!found && run < rank && rank <= run + c[b]) {
                digit = lane * 8 + b; before = run; inbin = c[b]; found = true;
            }
            run += c[b];
        }
    }
    digit = __shfl_sync(KNNG_FULL_MASK, digit, owner);
    before = __shfl_sync(KNNG_FULL_MASK, before, owner);
    inbin = __shfl_sync(KNNG_FULL_MASK, inbin, owner);
    if (lane == 0) {
        s.prefix |= (unsigned long long)digit << shift;
        s.mask |= 0xFFull << shift;
        s.rank -= (int)before;
        if ((uint32_t)s.rank == inbin || shift == 0) {
            s.done = 1;
            s.thr = s.prefix | (shift ? ((1ull << shift) - 1) : 0ull);
        }
        st[e] = s;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) big_count_kernel(int64_t n, int S, int nchunks, const Chunk* __restrict__ chunks,
                                                       const uint32_t* __restrict__ keys,
                                                       const int32_t* __restrict__ perm,
                                                       const SelState* __restrict__ st, int32_t* cnt)
{
    __shared__ int sh[33];
    const Chunk c = chunks[blockIdx.x];
    const int t = blockIdx.y;
    const unsigned long long thr = st[(int64_t)t * S + c.node].thr;
    const int64_t base = (int64_t)t * n + c.start;
    int v = 0;
    for (int e = threadIdx.x; e < c.len; e += NT) {
        const unsigned long long kv = ((unsigned long long)keys[base + e] << 32) | (uint32_t)perm[base + e];
        v += kv <= thr;
    }
    int total;
    block_excl_scan<NT>(v, sh, &total);
    if (threadIdx.x == 0) cnt[(int64_t)t * nchunks + blockIdx.x] = total;
}

// One block per (node, tree): exclusive scan of the node's chunk counts
// (in place: counts in, left-destination offsets out), NT chunks at a time.
// A node's chunks are contiguous in the level's chunk list; its first and
// its end are found by bisection.
template <int NT>
__global__ void __launch_bounds__(NT) big_base_kernel(int S, int nchunks, const Chunk* __restrict__ chunks,
                                                      int32_t* cnt_to_base)
{
    __shared__ int sh[33];
    const int s = blockIdx.x, t = blockIdx.y;
    auto first_of = [&](int node) {
        int lo = 0, hi = nchunks;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (chunks[mid].node < node) lo = mid + 1; else hi = mid;
        }
        return lo;
    };
    const int c_beg = first_of(s), c_end = first_of(s + 1);
    int32_t* row = cnt_to_base + (int64_t)t * nchunks;
    int run = 0;
    for (int c0 = c_beg; c0 < c_end; c0 += NT) {
        const int c = c0 + threadIdx.x;
        const int v = c < c_end ? row[c] : 0;
        int total;
        const int pre = block_excl_scan<NT>(v, sh, &total);
        if (c < c_end) row[c] = run + pre;
        run += total;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) big_scatter_kernel(int64_t n, int S, int nchunks, const Chunk* __restrict__ chunks,
                                                         const SplitNode* __restrict__ nodes,
                                                         const uint32_t* __restrict__ keys,
                                                         const int32_t* __restrict__ perm_cur,
                                                         const SelState* __restrict__ st,
                                                         const int32_t* __restrict__ lbase_arr,
                                                         int32_t* perm_nxt, int32_t* node_pos, int32_t* pos_of,
                                                         int32_t* node_of, int id_mode, const int* xb_bad)
{
    __shared__ unsigned long long k64[kChunk];
    __shared__ int sh[33];
    const Chunk c = chunks[blockIdx.x];
    const int t = blockIdx.y;
    const SplitNode nd = nodes[c.node];
    const unsigned long long thr = st[(int64_t)t * S + c.node].thr;
    const int64_t row = (int64_t)t * n;
    for (int e = threadIdx.x; e < c.len; e += NT)
        k64[e] = ((unsigned long long)keys[row + c.start + e] << 32) | (uint32_t)perm_cur[row + c.start + e];
    __syncthreads();
    const int32_t lb = lbase_arr[(int64_t)t * nchunks + blockIdx.x];
    const int32_t before = c.start - nd.off;
    stable_scatter<NT>(k64, c.len, thr, nd.off + lb, nd.off + nd.size / 2 + (before - lb), nd.childL,
                       nd.childR, perm_nxt + row, node_pos + row, pos_of + row, node_of + row,
                       want_id_maps(id_mode, xb_bad), sh);
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
// Tensor map of byte rows for the gather4 projection: n rows of ld bytes,
// boxes of 144 bytes x one row.  False when the CUDA driver's encoder or the
// encoding is unavailable (the projection then loads the rows itself).
static bool rows_tensor_map(CUtensorMap* map, const void* base, int64_t ld, int64_t n)
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    if (!fn || (uintptr_t)base % 16 != 0 || ld % 16 != 0 || n >= ((int64_t)1 << 31)) return false;
    const cuuint64_t gdim[2] = {(cuuint64_t)ld, (cuuint64_t)n};
    const cuuint64_t gstride[1] = {(cuuint64_t)ld};
    const cuuint32_t box[2] = {(cuuint32_t)kTmaRow, 1};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), gdim, gstride, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static inline int grid_for(int64_t work, int per_block, int cap)
{
    int64_t b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

cudaError_t run_partition(const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                          uint64_t seed, int32_t* perm_out, Arena& ar, cudaStream_t st, const LearnedFeat* lf,
                          int t0, const PcaOpt* pca, int* err)
{
    const int64_t n = x.n;
    const int d_pad = (x.d + 3) & ~3;
    const int S_max = std::max(P.max_nodes, 1);
    int32_t* perm_a = ar.take<int32_t>((size_t)T * n);
    int32_t* perm_b = ar.take<int32_t>((size_t)T * n);
    int32_t* pos_of = ar.take<int32_t>((size_t)T * n);
    int32_t* node_of = ar.take<int32_t>((size_t)T * n);
    int32_t* node_pos = ar.take<int32_t>((size_t)T * n);
    uint32_t* keys = ar.take<uint32_t>((size_t)T * n);
    float* dirs = ar.take<float>((size_t)T * S_max * d_pad);
    const int S_big = std::max(P.max_big_nodes, 1);
    SelState* sel = ar.take<SelState>((size_t)T * S_big);
    uint32_t* ghist = ar.take<uint32_t>((size_t)T * S_big * 256);
    int32_t* cnt = ar.take<int32_t>((size_t)T * std::max(P.max_chunks, 1));
    uint32_t* rmin = nullptr;
    uint32_t* rmax = nullptr;
    if (lf && lf->C > 0) {
        rmin = ar.take<uint32_t>((size_t)T * S_max);
        rmax = ar.take<uint32_t>((size_t)T * S_max);
    }
    if (!ar.base) return cudaSuccess;  // measuring only

    const int sms = num_sms();
    const int gcap = sms * 32;
    // byte input laid out for the node-major projection (16-byte aligned,
    // padded rows)
    const bool u8_nm_ok =
        x.dtype == kDtU8 && ((uintptr_t)x.X % 16 == 0) && (x.ld % 16 == 0) && (x.d % 16 == 0);
    // rows of at most 128 bytes for the node-major projection: gathered by
    // the tensor memory accelerator when their tensor map encodes
    CUtensorMap rows_map;
    bool tma_rows = false;
    if (((x.d + 15) & ~15) <= 128) {
        if (u8_nm_ok) tma_rows = rows_tensor_map(&rows_map, x.X, x.ld, n);
        else if (x.dtype == kDtF32 && x.Xb) tma_rows = rows_tensor_map(&rows_map, x.Xb, x.ldb, n);
    }
    init_perm_kernel<<<grid_for((int64_t)T * n, 256, gcap), 256, 0, st>>>(n, T, -1, perm_a, pos_of, node_of, node_pos);
    note_launches(1);
    if (!P.levels.empty()) {
        // slices of the roots, about 8 blocks per SM over all roots and trees
        const int64_t roots = (int64_t)P.levels[0].nnodes * T;
        const int slices = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8 / std::max<int64_t>(roots, 1),
                                                                       (n + 255) / 256));
        init_root_nodes_kernel<<<dim3(slices, P.levels[0].nnodes, T), 256, 0, st>>>(n, dp.nodes, node_of, node_pos);
        note_launches(1);
    }
    int32_t* cur = perm_a;
    int32_t* nxt = perm_b;
    for (size_t lvl = 0; lvl < P.levels.size(); ++lvl) {
        const LevelPlan& L = P.levels[lvl];
        const SplitNode* nodes = dp.nodes + L.node_base;
        const int S = L.nnodes;
        const bool learned = lf && lf->Z && (int)lvl < lf->C;
        LevelFeat lv{};
        if (learned) {
            lv.Z = lf->Z;
            lv.C = lf->C;
            for (int t = 0; t < T && t0 + t < 32; ++t) lv.ft.f[t] = lf->feat[t0 + t][lvl];
            lv.rmin = rmin;
            lv.rmax = rmax;
            lv.frange = lf->frange;
            lv.tau = lf->tau;
            cudaMemsetAsync(rmin, 0xFF, sizeof(uint32_t) * (size_t)T * S, st);
            cudaMemsetAsync(rmax, 0, sizeof(uint32_t) * (size_t)T * S, st);
            node_feature_range_kernel<<<grid_for((int64_t)T * n, 256, gcap), 256, 0, st>>>(n, T, lf->Z, lf->C, lv.ft,
                                                                                         node_pos, cur, S, rmin,
                                                                                         rmax);
            note_launches(1);
        }
        gen_dirs_kernel<<<grid_for((int64_t)T * S * (d_pad / 4), 256, gcap), 256, 0, st>>>(
            dirs, T, S, x.d, d_pad, nodes, (uint32_t)lvl, seed, (uint32_t)t0);
        note_launches(1);
        if (pca && pca->on) {
            // principal directions of the nodes' samples, from the random ones
            const cudaError_t e = run_pca_dirs(x, T, S, nodes, cur, d_pad, (uint32_t)lvl, seed, t0, dirs, pca->out,
                                               pca->stride, st);
            if (e != cudaSuccess) return e;
        }
        const int pgrid = grid_for(n * 32, 256, sms * 16);
        // byte rows with 16-byte aligned, padded rows go node-major: the
        // internal exact byte copy of float rows (decided on the device), or
        // byte input laid out that way
        const bool copy_nm = !learned && x.dtype == kDtF32 && x.Xb != nullptr;
        const bool u8_nm = !learned && u8_nm_ok;
        const int bgrid = grid_for((int64_t)T * n, 256, sms * 16);
        if (copy_nm || u8_nm) {
            const RowLoader<kDtU8> rb = u8_nm ? RowLoader<kDtU8>{x.X, x.ld, x.d, true}
                                              : RowLoader<kDtU8>{x.Xb, x.ldb, x.d, true};
            if (tma_rows && x.d == 128)
                project_bytes_tma_kernel<true><<<bgrid, 256, 0, st>>>(rows_map, x.d, x.xb_bad, u8_nm, n, T, dirs, S,
                                                                      d_pad, cur, node_pos, keys, err);
            else if (tma_rows)
                project_bytes_tma_kernel<false><<<bgrid, 256, 0, st>>>(rows_map, x.d, x.xb_bad, u8_nm, n, T, dirs, S,
                                                                       d_pad, cur, node_pos, keys, err);
            else if (x.d == 128)
                project_bytes_kernel<true, true><<<bgrid, 256, 0, st>>>(rb, x.xb_bad, u8_nm, n, T, dirs, S, d_pad, cur,
                                                                        node_pos, keys);
            else if (((x.d + 15) & ~15) <= 128)
                project_bytes_kernel<true, false><<<bgrid, 256, 0, st>>>(rb, x.xb_bad, u8_nm, n, T, dirs, S, d_pad,
                                                                         cur, node_pos, keys);
            else
                project_bytes_kernel<false, false><<<bgrid, 256, 0, st>>>(rb, x.xb_bad, u8_nm, n, T, dirs, S, d_pad,
                                                                          cur, node_pos, keys);
            note_launches(1);
        }
        if (!u8_nm) {
            auto project = [&](auto dt) {
                constexpr int kDT = decltype(dt)::value;
                RowLoader<kDT> rl{x.X, x.ld, x.d, x.vec};
                const RowLoader<kDtU8> rb{x.Xb, x.ldb, x.d, true};
                if (learned)
                    project_kernel<kDT, true><<<pgrid, 256, 0, st>>>(rl, rb, x.xb_bad, copy_nm, n, T, dirs, S, d_pad,
                                                                     node_of, pos_of, keys, lv);
                else
                    project_kernel<kDT, false><<<pgrid, 256, 0, st>>>(rl, rb, x.xb_bad, copy_nm, n, T, dirs, S, d_pad,
                                                                      node_of, pos_of, keys, lv);
            };
            if (x.dtype == kDtF16) project(std::integral_constant<int, kDtF16>{});
            else if (x.dtype == kDtU8) project(std::integral_constant<int, kDtU8>{});
            else project(std::integral_constant<int, kDtF32>{});
            note_launches(1);
        }
        // which maps by id the scatter keeps: the next level's projection
        // reads them unless it goes node-major (byte rows), and none follows
        // the last level
        int id_mode = 1;
        if (lvl + 1 >= P.levels.size()) id_mode = 0;
        else if (lf && lf->Z && (int)lvl + 1 < lf->C) id_mode = 1;
        else if (u8_nm_ok) id_mode = 0;
        else if (x.dtype == kDtF32 && x.Xb != nullptr) id_mode = 2;
        // leaves of this level keep their positions: start from a copy,
        // unless the level's split nodes cover every position
        int64_t covered = 0;
        for (int s = 0; s < S; ++s) covered += P.nodes[L.node_base + s].size;
        if (covered < n) cudaMemcpyAsync(nxt, cur, sizeof(int32_t) * (size_t)T * n, cudaMemcpyDeviceToDevice, st);
        if (L.nbig < S) {
            constexpr int NT = 512;
            const size_t smem = sizeof(unsigned long long) * (size_t)L.max_small;
            static bool attr = false;
            if (!attr) {
                cudaError_t e = cudaFuncSetAttribute(split_small_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)(sizeof(unsigned long long) * kSmallCap));
                if (e != cudaSuccess) return e;
                attr = true;
            }
            split_small_kernel<NT><<<dim3(S - L.nbig, T), NT, smem, st>>>(n, nodes + L.nbig, keys, cur, nxt, node_pos,
                                                                         pos_of, node_of, id_mode, x.xb_bad);
            note_launches(1);
        }
        if (L.nbig > 0) {
            constexpr int NT = 256;
            const int SB = L.nbig;
            const Chunk* chunks = dp.chunks + L.chunk_base;
            const int NC = L.nchunks;
            big_init_kernel<<<(SB * T + 255) / 256, 256, 0, st>>>(SB, T, nodes, sel);
            note_launches(1);
            cudaMemsetAsync(ghist, 0, sizeof(uint32_t) * (size_t)T * SB * 256, st);
            for (int shift = 56; shift >= 0; shift -= 8) {
                big_hist_kernel<NT><<<dim3(NC, T), NT, 0, st>>>(n, shift, SB, chunks, keys, cur, sel, ghist);
                note_launches(1);
                big_pick_kernel<<<dim3(SB, T), 32, 0, st>>>(shift, SB, sel, ghist);
                note_launches(1);
            }
            big_count_kernel<NT><<<dim3(NC, T), NT, 0, st>>>(n, SB, NC, chunks, keys, cur, sel, cnt);
            note_launches(1);
            big_base_kernel<256><<<dim3(SB, T), 256, 0, st>>>(SB, NC, chunks, cnt);
            note_launches(1);
            big_scatter_kernel<NT><<<dim3(NC, T), NT, 0, st>>>(n, SB, NC, chunks, nodes, keys, cur, sel, cnt, nxt,
                                                               node_pos, pos_of, node_of, id_mode, x.xb_bad);
            note_launches(1);
        }
        std::swap(cur, nxt);
    }
    cudaMemcpyAsync(perm_out, cur, sizeof(int32_t) * (size_t)T * n, cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

}  // namespace knng
