// Host-side plan of a partition tree and the launchers of every stage.
// Not part of the public ABI (include/knng.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/knng.h"

#include <algorithm>
#include <map>
#include <string>
#include <vector>

namespace knng {

// A node that is split at its level.  childL/childR index the split nodes of
// the next level, or are -1 when that child is a leaf.
struct SplitNode {
    uint32_t v;     // node number within its level (children are 2v, 2v+1)
    int32_t off;    // first position of the node in the permutation
    int32_t size;   // number of points (> leaf size)
    int32_t childL;
    int32_t childR;
    int32_t pad[3];
};

// A slice of a large node, processed by one block in the multi-block split.
struct Chunk {
    int32_t node;   // index into the level's split nodes
    int32_t start;  // absolute position of the slice
    int32_t len;
    int32_t first;  // index of the node's first chunk in the level's chunk list
};

struct SelState {
    unsigned long long prefix;
    unsigned long long mask;
    unsigned long long thr;
    int32_t rank;
    int32_t done;
};

constexpr int kSmallCap = 8192;    // nodes up to this size split in one block
constexpr int kChunk = 4096;       // slice size of the multi-block split
constexpr int kMaxLeaf = 512;      // largest leaf size g
constexpr int kMaxK = 64;
constexpr int kMaxT = 32;

// The split nodes of one level: the nbig nodes larger than kSmallCap come
// first (split by the multi-block path), the others after them (one block
// each).
struct LevelPlan {
    int64_t node_base;   // offset of this level's SplitNode array in the plan table
    int32_t nnodes;
    int32_t nbig;
    int32_t max_small;   // largest node split by one block (0 if none)
    int64_t chunk_base;  // offset of this level's Chunk array (big nodes)
    int32_t nchunks;
};

// Shape of every tree over n points with leaf size g (shared by all trees),
// or of a forest: one tree per root segment (independent point sets stored
// back to back), with node numbers local to each tree.
struct TreePlan {
    int64_t n = -1;
    int g = -1;
    std::vector<int64_t> roots;    // root sizes (one root for a single set)
    std::vector<LevelPlan> levels;
    std::vector<SplitNode> nodes;  // all levels, concatenated
    std::vector<Chunk> chunks;     // large levels, concatenated
    std::vector<int32_t> leaf_off; // nleaves + 1
    int32_t max_nodes = 0;         // widest level
    int32_t max_chunks = 0;
    int32_t max_big_nodes = 0;     // widest level split by the multi-block path
    int32_t max_leaf = 0;          // largest leaf
};

void make_tree_plan(int64_t n, int g, TreePlan& plan);
void make_forest_plan(const std::vector<int64_t>& roots, int g, TreePlan& plan);

// Device copy of a TreePlan.
struct DevPlan {
    const SplitNode* nodes = nullptr;
    const Chunk* chunks = nullptr;
    const int32_t* leaf_off = nullptr;
};

// Bump allocator over the handle's workspace.  With base == nullptr it only
// measures.
struct Arena {
    char* base = nullptr;
    size_t off = 0;
    template <class T>
    T* take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

struct XDesc {
    const void* X;
    int dtype;  // 0 f32, 1 f16, 2 u8
    int64_t n;
    int d;
    int64_t ld;
    bool vec;
    // Optional byte copy of float rows (n rows of ldb bytes) and a device word
    // that stays 0 when every entry of X is an integer in [0, 255] (d <= 256):
    // the copy then holds exactly the same values, and the row-gathering
    // kernels (projection, propagation) read it instead of X.
    const uint8_t* Xb = nullptr;
    int64_t ldb = 0;
    const int* xb_bad = nullptr;
};

// Learned split features: Z[n][C] (FP32) and, per tree t, the feature used
// at level l < C (feat[t][l], a permutation of 0..C-1).
// A node splits along its learned feature only while that feature still
// varies inside the node: range within the node > tau x range over all
// points; otherwise (a feature that has saturated into a constant there) it
// splits along its random direction.
struct LearnedFeat {
    const float* Z = nullptr;
    int C = 0;
    int feat[32][32] = {};
    float tau = 0.02f;
    const float* frange = nullptr;  // device [C]: max - min of each feature over all points
};
cudaError_t run_feature_range(const float* Z, int64_t n, int C, uint32_t* scratch2C, float* frange, cudaStream_t st);
// Per-tree feature order from Philox (Fisher-Yates), a function of (seed, t).
void learned_feature_order(uint64_t seed, int T, int C, LearnedFeat& lf);

// ---- stages (each carves its scratch from the arena) -------------------
// Principal-direction splits (Sec. 3.4): on, and an optional output of the
// directions, tree t's node (level, v) at out[t * stride + (2^level - 1 + v) * d].
struct PcaOpt {
    bool on = false;
    float* out = nullptr;
    int64_t stride = 0;
};
cudaError_t run_pca_dirs(const XDesc& x, int T, int S, const SplitNode* nodes, const int32_t* cur, int dp,
                         uint32_t level, uint64_t seed, int t0, float* dirs, float* out, int64_t out_tree_stride,
                         cudaStream_t st);

// Trees t0 .. t0 + T - 1 (perm_out[T][n]).
cudaError_t run_partition(const XDesc& x, const TreePlan& plan, const DevPlan& dp, int T,
                          uint64_t seed, int32_t* perm_out, Arena& ar, cudaStream_t st,
                          const LearnedFeat* lf = nullptr, int t0 = 0, const PcaOpt* pca = nullptr,
                          int* err = nullptr);

cudaError_t run_leaf_knn_f32(const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                             const int32_t* perm, int k, int kp, int32_t* ids, float* dists,
                             cudaStream_t st);

// Tile choices of the tensor-core leaf kernel for one problem shape:
// pipeline stages S and epilogue row-group height RG (32, 64 or 128).
struct TcTile {
    int S = 0;
    int RG = 0;
};
// Shape key of the tensor-core leaf kernel: precision, padded row bytes and
// the widest leaf (MMA N) -- the quantities its geometry depends on.
struct TcKey {
    int prec, row_bytes, n_load;
    bool operator<(const TcKey& o) const
    {
        if (prec != o.prec) return prec < o.prec;
        if (row_bytes != o.row_bytes) return row_bytes < o.row_bytes;
        return n_load < o.n_load;
    }
};
TcKey tc_key(const TreePlan& P, int d, int prec);
// Candidate tiles for a shape (valid for its shared-memory budget).
std::vector<TcTile> tc_candidates(const TreePlan& P, int d, int prec);

// Staged FP32 rescoring of reduced-precision leaf candidates (one CTA per
// tree and leaf; the leaf's rows stream through shared memory in 32-entry
// slices): FP32 rows, 16-byte aligned, k' <= 32, leaves of at most 512.
bool leaf_rescore_staged_ok(const XDesc& x, int kp, int max_leaf);
cudaError_t run_leaf_rescore_staged(const XDesc& x, const TreePlan& P, const DevPlan& dp, int T,
                                    const int32_t* perm, const uint8_t* leaf_exact, const uint16_t* cand, int kp,
                                    int k, int32_t* ids, float* dists, cudaStream_t st);

// all_exact (nullable): cleared by every leaf whose distances are not all
// exact (its list is then not the exact k best of the leaf).
// wait_cycles: limit of the waits on the TMA copies and on the MMAs' release
// of a pipeline stage (0: about one second); a CTA that gives up sets *err,
// then waits for its own copies and MMAs under the long limit and returns.
cudaError_t run_leaf_knn_tc(const XDesc& x, const TreePlan& P, const DevPlan& dp, int T, const int32_t* perm,
                            int k, int kp, int prec, int32_t* ids, float* dists, int* err, Arena& ar,
                            cudaStream_t st, const TcTile* tile = nullptr, int* all_exact = nullptr,
                            long long wait_cycles = 0);

// tmask (nullable, T <= 8): per output entry, the trees whose lists held
// it, when *all_exact != 0 (every leaf list exact); zeros otherwise.
cudaError_t run_merge(int64_t n, int T, int k, const int32_t* ids_in, const float* d_in,
                      int32_t* ids, float* dists, cudaStream_t st, uint8_t* tmask = nullptr,
                      const int* all_exact = nullptr);
// One more division into the running graph: lists (ia, da) and (ib, db) ->
// the k best of both; counts[0] += entries not in a, counts[1] += entries.
cudaError_t run_merge_add(int64_t n, int k, const int32_t* ia, const float* da, const int32_t* ib, const float* db,
                          int32_t* ids, float* dists, unsigned long long* counts, cudaStream_t st);
// Budgeted best-first propagation pass (Sec. 3.2), synchronous.
cudaError_t run_propagate_best_first(const XDesc& x, int k, int budget, const int32_t* order, const int32_t* ids_in,
                                     int32_t* ids, float* dists, cudaStream_t st);

// Byte copy of float rows (see XDesc::Xb); *bad is set when an entry is not
// an integer in [0, 255].  *bad must be 0 on entry.
cudaError_t run_byte_copy(const XDesc& x, uint8_t* Xb, int64_t ldb, int* bad, cudaStream_t st);

// Cosine metric: rows scaled to unit length (FP32, out rows of ldo floats),
// and an in-place scale of n floats.
cudaError_t run_normalize_rows(const XDesc& x, float* out, int64_t ldo, cudaStream_t st);
cudaError_t run_scale(float* v, int64_t cnt, float f, cudaStream_t st);

// Pairwise-updating offers of one propagation round (see propagate.cu):
// offer (target c, packed (dist, source p)) pairs, at most cap of them, a
// running count, per-target counts, and the error word (2 = overflow).
struct PairOffers {
    int32_t* tgt = nullptr;
    uint64_t* key = nullptr;
    unsigned long long* count = nullptr;
    int32_t* per_tgt = nullptr;
    unsigned long long cap = 0;
    int* err = nullptr;
};

// One synchronous propagation round.  flags_in (nullable = every entry new)
// marks, per point, the list entries that were not in the previous round's
// list; flags_out (nullable) receives the same for the output lists.
// tmask_in (nullable): the merge's tree masks of the input lists (exact
// leaves only); a neighbour's entry that shares a tree with p's entry for
// that neighbour is skipped.
// stats (nullable): stats[0] += candidate rows scored, stats[1] += slots of
// the neighbours' lists loaded (what the round actually reads).
cudaError_t run_propagate(const XDesc& x, int k, const int32_t* order, const int32_t* ids_in, const float* d_in,
                          const unsigned long long* flags_in, int32_t* ids, float* dists,
                          unsigned long long* flags_out, cudaStream_t st, const PairOffers* offers = nullptr,
                          const uint8_t* tmask_in = nullptr,
                          unsigned long long* stats = nullptr);

// Scratch of a pairwise round: offers (cap entries), per-target counts and
// offsets, forward lists.  pairwise_bytes() sizes it.
struct PairScratch {
    PairOffers po;
    int64_t* off = nullptr;       // [n + 1]
    int64_t* bsum = nullptr;      // scan block sums
    uint64_t* sorted = nullptr;   // [cap] offers grouped by target
    int32_t* fwd_i = nullptr;     // [n][k]
    float* fwd_d = nullptr;       // [n][k]
};
void pairwise_take(Arena& a, int64_t n, int k, PairScratch& s);
cudaError_t run_propagate_pairwise(const XDesc& x, int k, const int32_t* order, const int32_t* ids_in,
                                   const float* d_in, const unsigned long long* flags_in, int32_t* ids, float* dists,
                                   unsigned long long* flags_out, const PairScratch& s, int* err, cudaStream_t st);

cudaError_t run_exact_knn(const XDesc& x, const int32_t* queries, int nq, int k, int32_t* ids,
                          float* dists, cudaStream_t st);

// One set of a batched build, as seen by the output scatter.
struct BatchSet {
    int64_t off;  // first global point id of the set
    int64_t n;
    int32_t* ids;
    float* dists;
};
cudaError_t run_scatter_batch(int64_t ng, int k, const BatchSet* sets, int nsets, const int32_t* gi,
                              const float* gd, cudaStream_t st);

// Split-feature network of the learned partitioner (parameters packed as
// W1[H][d] | b1[H] | W2[C][H] | b2[C], FP32, on the device).
struct MlpModel {
    int device = 0;
    int d = 0, H = 0, C = 0;
    int64_t count = 0;       // packed parameters: W1 | b1 | W2 | b2
    float* w = nullptr;      // device, packed
    float* g = nullptr;      // gradient
    float* am = nullptr;     // Adam moments
    float* av = nullptr;
    int64_t adam_t = 0;
    // training buffers (grown on demand)
    int cap_rows = 0;
    float* Xb = nullptr;
    float* A = nullptr;
    float* Hh = nullptr;
    float* Z = nullptr;
    float* dZ = nullptr;
    float* loss = nullptr;
    // BF16 inference images (swizzled operand layouts), rebuilt when stale
    void* img = nullptr;
    bool img_stale = true;
    float* W1() const { return w; }
    float* b1() const { return w + (int64_t)H * d; }
    float* W2() const { return b1() + H; }
    float* b2() const { return W2() + (int64_t)C * H; }
};
MlpModel* mlp_model(knng_mlp* o);
// z = W2 GELU(W1 x + b1) + b2 for every point, BF16 on the tensor cores.
cudaError_t run_mlp_forward(MlpModel& M, const XDesc& x, float* Z, int* err, cudaStream_t st);

int num_sms();

// Count of kernels this library has launched (all handles, all devices).
void note_launches(int count);
unsigned long long launch_count();

}  // namespace knng
