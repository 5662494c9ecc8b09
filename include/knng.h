/*
 * knng.h -- C ABI of the GB300 k-NN graph library.
 *
 * The library builds an approximate k-nearest-neighbour graph by the method of
 * Wang, Wang, Zeng, Tu, Gan and Li, "Scalable k-NN graph construction"
 * (arXiv:1307.7852): T random hierarchical divisions of the points (Sec. 3.1),
 * an exact brute-force graph inside every leaf subset (Sec. 3.1), the union of
 * the T base graphs keeping the k nearest (Sec. 3.1), and neighbourhood
 * propagation (Sec. 3.2; the first-order form of Theorem 1).
 *
 * Conventions shared by every entry point:
 *  - Pointers named X, ids, dists, perm, *_in are DEVICE pointers (cudaMalloc,
 *    torch tensors, ...), owned by the caller; the library never frees them.
 *    Entry points whose name ends in _host take HOST pointers instead.
 *  - X is row-major: point i starts at element i*ld; ld >= d.  dtype is
 *    KNNG_DTYPE_F32 (float), KNNG_DTYPE_F16 (IEEE half) or KNNG_DTYPE_U8
 *    (unsigned bytes, e.g. SIFT descriptors); F16 and U8 entries are widened
 *    exactly to float, and every result is the one for the equal float rows.
 *  - Graph outputs are ids[n][k] (int32) and dists[n][k] (float): the
 *    neighbours of point i in row i, ordered by (distance, id) ascending,
 *    never containing i, without duplicates.  A distance is the SQUARED
 *    Euclidean distance (it ranks like the Euclidean distance of Def. 1).
 *    Rows are padded with id -1 / distance +inf only when fewer than k other
 *    candidates exist.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *    work is enqueued on it; calls return after enqueueing, except those
 *    ending in _host, which return after the results are on the host.
 *  - Return value: KNNG_OK (0) or a negative KNNG_ERR_* code.  Nothing aborts
 *    and nothing throws across the ABI.  knng_last_error() describes the last
 *    failure of a handle.
 *  - A handle owns a device workspace, grown on demand with the stream-ordered
 *    allocator; calls on one handle must not run concurrently from several
 *    host threads.
 */
#ifndef KNNG_H
#define KNNG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define KNNG_OK 0
#define KNNG_ERR_INVALID_ARG (-1) /* a size, pointer or parameter is out of range */
#define KNNG_ERR_UNSUPPORTED (-2) /* valid request the library does not serve     */
#define KNNG_ERR_OOM (-3)         /* device workspace allocation failed          */
#define KNNG_ERR_CUDA (-4)        /* a CUDA runtime call or launch failed        */
#define KNNG_ERR_TIMEOUT (-5)     /* a bounded device wait gave up               */
#define KNNG_ERR_INTERNAL (-6)
#define KNNG_ERR_LIMIT (-7)       /* request exceeds a fixed capacity (see knng_propagate_noalloc) */

/* ---- enumerations ---------------------------------------------------- */
#define KNNG_DTYPE_F32 0
#define KNNG_DTYPE_F16 1
#define KNNG_DTYPE_U8 2

/* Precision of the leaf candidate stage.  The leaf top-k' is chosen on
 * distances computed from rows at this precision, then every candidate is
 * rescored in FP32 by direct differences and the k best are kept. */
#define KNNG_PREC_FP32 0
#define KNNG_PREC_BF16 1
#define KNNG_PREC_FP8E4M3 2

#define KNNG_PART_RANDOM 0  /* Philox random directions (App. after Lemma 1)                  */
#define KNNG_PART_PCA 1     /* random principal directions (Sec. 3.4): see knng_partition_pca */
#define KNNG_PART_FEATURES 2 /* knng_build_learned only: per-level learned features              */
#define KNNG_PART_FEATURES_PCA 3 /* the same with principal directions where a feature is flat   */

/* Distance.  L2: the squared Euclidean distance.  COSINE: 1 - cos of the
 * angle between two rows (App. after Lemma 1: random projections partition
 * for the cosine distance too).  For COSINE the rows are first scaled to
 * unit length in FP32 (knng_normalize_rows) and the method runs on the unit
 * rows u, whose |u - v|^2 / 2 is 1 - cos; a zero row stays zero (distance
 * 1/2 to every unit row).  The scaled copy takes n * round_up(d, 4) floats
 * of the workspace. */
#define KNNG_METRIC_L2 0
#define KNNG_METRIC_COSINE 1

/* Propagation scheme of the prop_rounds rounds.
 * FIRST_ORDER (Theorem 1): every point takes the k best of its list and its
 *   neighbours' lists.
 * BEST_FIRST (Sec. 3.2): every point visits its neighbours, then repeatedly
 *   the not yet visited neighbours of the nearest visited point it has not
 *   expanded (a priority queue keyed by the FP32 distance, ties by id), until
 *   `budget` points were visited or nothing is left; it keeps the k best
 *   visited.  Each round reads a frozen snapshot of the lists.
 * PAIRWISE (Sec. 3.4): FIRST_ORDER in which every candidate pair (p, c) is
 *   also offered the other way: p enters c's list if it is among c's k best.
 *   Offers are buffered, 4 per list entry; knng_sync reports
 *   KNNG_ERR_LIMIT if a round had more (the lists stay valid). */
#define KNNG_PROP_FIRST_ORDER 0
#define KNNG_PROP_BEST_FIRST 1
#define KNNG_PROP_PAIRWISE 2

/* ---- parameters ------------------------------------------------------ */
typedef struct knng_params {
    int32_t k;            /* neighbours per point, 1 <= k <= 64, k < leaf_size/2     */
    int32_t T;            /* random divisions (trees), 1 <= T <= 32 (Sec. 3.1's M)   */
    int32_t leaf_size;    /* g: a node with at most g points is a leaf, 2..512 (Sec. 3.1) */
    int32_t prop_rounds;  /* R: first-order propagation rounds, 0..16 (Sec. 3.2)     */
    uint64_t seed;        /* key of the Philox directions; same seed -> same trees   */
    int32_t precision;    /* KNNG_PREC_*                                             */
    int32_t rescore_mult; /* k' = rescore_mult * k candidates per leaf row, 1..4     */
    int32_t partitioner;  /* KNNG_PART_RANDOM or KNNG_PART_PCA (d <= 1024)           */
    int32_t metric;       /* KNNG_METRIC_L2 or KNNG_METRIC_COSINE                    */
    int32_t propagation;  /* KNNG_PROP_*                                             */
    int32_t budget;       /* KNNG_PROP_BEST_FIRST: points visited per point, k..512  */
    float r_stop;         /* > 0: divisions are added one by one until the effective
                             rate r_m of the last one is below r_stop (Sec. 4 uses
                             0.05), at most T; 0: exactly T divisions            */
    int32_t reserved;     /* must be 0                                               */
} knng_params;

typedef struct knng_handle knng_handle;

/* ---- handle ---------------------------------------------------------- */
/* Creates a handle bound to CUDA device `device` (made current for the call).
 * *out receives the handle; returns KNNG_ERR_INVALID_ARG for a bad device. */
int knng_create(knng_handle** out, int32_t device);
/* Frees the workspace (after synchronising the device) and the handle. */
int knng_destroy(knng_handle* h);
/* Static description of a status code; never NULL. */
const char* knng_status_string(int32_t status);
/* Message of the last failure on h ("" if none); valid until the next call. */
const char* knng_last_error(const knng_handle* h);

/* Synchronises `stream` and reports device-side failures of earlier calls on
 * h: KNNG_ERR_TIMEOUT if a bounded wait inside a kernel gave up (the outputs
 * of those calls are then invalid); the flag is cleared. */
int knng_sync(knng_handle* h, void* stream);

/* Limit, in SM clock cycles, of the tensor-core leaf kernel's waits for its
 * TMA copies and for the MMAs to release a pipeline stage, for later calls
 * on h (0, the default: 2e9 cycles, about one second).  A CTA whose wait
 * runs out records KNNG_ERR_TIMEOUT for knng_sync, waits (under the one-second
 * limit) for the copies and MMAs it started, frees its tensor memory and
 * returns; the context stays usable.  A small limit makes waits on copies
 * that do complete give up -- a way to exercise that path.  cycles < 0:
 * KNNG_ERR_INVALID_ARG.  No counterpart in the paper. */
int knng_set_wait_limit(knng_handle* h, int64_t cycles);

/* Counters of what the first-order propagation rounds read (Sec. 3.2;
 * measurement of the rounds' real traffic, with the exact skips of pairs
 * that cannot enter a list).  counters: device array of 2 * rounds uint64,
 * zeroed by the caller; while set, round r < rounds of every later
 * knng_build / knng_propagate call on h adds to counters[2r] the candidate
 * rows it scored and to counters[2r + 1] the slots of neighbours' lists it
 * loaded.  rounds = 0 (or counters NULL with rounds 0) turns counting off,
 * the default; counting adds one atomic per warp.  The array must outlive
 * the calls that use it.  No counterpart in the paper. */
int knng_set_propagation_counters(knng_handle* h, uint64_t* counters, int32_t rounds);

/* ---- tree shape (host only) ------------------------------------------ */
/* Every split halves a node of m points into floor(m/2) (left) and
 * ceil(m/2) (right) points, so the leaf layout of a tree depends on (n, g)
 * only and is shared by all trees.  knng_leaf_count writes the number of
 * leaves; knng_leaf_offsets writes the nleaves+1 start offsets of the leaves
 * (left to right) into the HOST array leaf_off. */
int knng_leaf_count(int64_t n, int32_t leaf_size, int64_t* nleaves);
int knng_leaf_offsets(int64_t n, int32_t leaf_size, int64_t* leaf_off);

/* ---- whole method ---------------------------------------------------- */
/* Builds the approximate k-NN graph of X[n][d] (Sec. 3): p->T divisions,
 * leaf graphs, merge, p->prop_rounds propagation rounds.  ids, dists: device
 * [n][k].  2 <= n < 2^31, 1 <= d <= 4096.
 * Float rows with d <= 256 are also checked on the device, in one pass, for
 * holding only integers 0..255 (descriptor data such as SIFT); if they do,
 * the projection and propagation read an exact byte copy of X kept in the
 * workspace (n * round_up(d, 16) bytes more).  The result does not change:
 * the copy holds the same values, and with d * 255^2 < 2^24 every FP32
 * distance between such rows is an exact integer. */
int knng_build(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
               const knng_params* p, int32_t* ids, float* dists, void* stream);
/* Same as knng_build with HOST X, ids and dists: copies X to the device,
 * builds, copies the graph back and synchronises `stream` before returning. */
int knng_build_host(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d,
                    int64_t ld, const knng_params* p, int32_t* ids, float* dists, void* stream);

/* ---- many independent point sets ----------------------------------------- */
/* One independent point set of a batch: X (device, row-major, rows of ld
 * elements) and its outputs ids/dists (device [n][k]). */
typedef struct knng_dataset {
    const void* X;
    int32_t dtype; /* KNNG_DTYPE_* */
    int32_t d;
    int64_t n;
    int64_t ld;
    int32_t* ids;
    float* dists;
} knng_dataset;

/* Builds the graphs of nsets independent point sets with the same
 * parameters (Sec. 3 applied to each set).  Every set gets exactly the graph
 * knng_build would produce for it alone.  Sets of equal (d, dtype) are
 * processed together: their trees form one forest whose roots are the sets,
 * so each stage is one launch for the whole group.  The first call with a
 * given batch (pointers, sizes, parameters) records the whole batch once as a
 * CUDA graph; later identical calls replay it with a single graph launch.
 * The first call synchronises `stream` (table upload); make it outside any
 * stream capture.  1 <= nsets <= 65536; per set the limits of knng_build. */
int knng_build_batched(knng_handle* h, int32_t nsets, const knng_dataset* sets, const knng_params* p,
                       void* stream);

/* ---- tile autotuning (tensor-core leaf kernel) --------------------------- */
/* Times the tensor-core leaf kernel (p->precision BF16 or FP8E4M3) on X with
 * every valid tile choice -- pipeline stages and epilogue row-group height --
 * and keeps the fastest in h for this problem shape (precision, padded row
 * length, widest leaf).  Later builds and batched builds on h of the same
 * shape use it; results do not depend on the choice, only speed.  Optional
 * outputs (may be NULL): the chosen stages, rows per group and its mean time
 * per leaf stage in ms.  Synchronises `stream`. */
int knng_autotune(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                  const knng_params* p, int32_t* stages, int32_t* rows_per_group, float* best_ms,
                  void* stream);
/* Writes / reads the tile choices of h as a text file (one shape per line). */
int knng_tune_save(knng_handle* h, const char* path);
int knng_tune_load(knng_handle* h, const char* path);

/* ---- stages ---------------------------------------------------------- */
/* Random divisions (Sec. 3.1; split rule of the appendix after Lemma 1).
 * perm: device int32 [T][n].  Row t lists the point ids of tree t leaf by
 * leaf, left to right, ids ascending inside each leaf (the canonical leaf
 * set; leaf boundaries from knng_leaf_offsets).  Tree t depends only on
 * (X, seed, t, leaf_size). */
int knng_partition(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                   int32_t T, int32_t leaf_size, uint64_t seed, int32_t* perm, void* stream);

/* Number of split levels of the tree shape of (n, g) (host only): the
 * depth L of the deepest split node + 1; the nodes of level l are numbered
 * v = 0 .. 2^l - 1 left to right. */
int knng_split_levels(int64_t n, int32_t g, int32_t* levels);

/* Random partition trees with principal-direction splits (Sec. 3.4, "Random
 * division"): every node of m > g points splits at the median along the
 * principal direction of points sampled from it.  Readings (the paper gives
 * no sizes): a node with m <= s_cap points uses all of them, otherwise
 * s_cap members chosen with replacement by Philox4x32-10 (counter (tree,
 * level | 2^30, node, r / 4), key seed; member index = word mod m, members in
 * ascending id order); s_cap = clamp(floor(40960 / d), 8, 128).  The
 * direction: at most min(8, d) Lanczos steps with full reorthogonalisation
 * on the FP32 covariance of the centred sample, started from the node's
 * random direction, stopping once beta <= 1e-4 * max alpha; the top Ritz
 * vector, unit length, largest-magnitude entry positive.  perm as in
 * knng_partition.  dirs_out (device, may be NULL): T x (2^L - 1) x d floats,
 * tree t's node (level, v) direction in row 2^level - 1 + v (rows of other
 * slots are left untouched); L from knng_split_levels.  d <= 1024. */
int knng_partition_pca(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, int32_t T,
                       int32_t g, uint64_t seed, int32_t* perm, float* dirs_out, void* stream);

/* Leaf graphs (Sec. 3.1): for every tree t and point i, the k nearest other
 * members of i's leaf.  perm: device [T][n] as written by knng_partition.
 * ids, dists: device [T][n][k] (row t*n+i is point i in tree t). */
int knng_leaf_knn(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                  int32_t T, int32_t leaf_size, const int32_t* perm, int32_t k,
                  int32_t precision, int32_t rescore_mult, int32_t* ids, float* dists,
                  void* stream);

/* Combination of base graphs (Sec. 3.1): for every point, the union of its T
 * lists (ids_in/dists_in device [T][n][k], each row ordered by (distance,
 * id)), duplicates removed by id, the k best kept.  ids, dists: [n][k]. */
int knng_merge(knng_handle* h, int64_t n, int32_t T, int32_t k, const int32_t* ids_in,
               const float* dists_in, int32_t* ids, float* dists, void* stream);

/* Neighbourhood propagation (Sec. 3.2, first-order form of Theorem 1):
 * `rounds` synchronous rounds; in each, every point p takes the k best of
 * its list and its neighbours' lists (without p), scoring new candidates by
 * exact FP32 distances.  ids_in/dists_in: device [n][k]; ids, dists: [n][k].
 * The input and output may not overlap. */
int knng_propagate(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                   int32_t k, int32_t rounds, const int32_t* ids_in, const float* dists_in,
                   int32_t* ids, float* dists, void* stream);

/* Best-first propagation with a visit budget (Sec. 3.2; see
 * KNNG_PROP_BEST_FIRST): `rounds` synchronous passes.  k <= budget <= 512.
 * ids_in: device [n][k]; ids, dists: [n][k], not overlapping the input. */
int knng_propagate_best_first(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                              int32_t k, int32_t budget, int32_t rounds, const int32_t* ids_in, int32_t* ids,
                              float* dists, void* stream);

/* First-order propagation with pairwise updating (Sec. 3.4; see
 * KNNG_PROP_PAIRWISE): `rounds` synchronous rounds.  Buffers as in
 * knng_propagate; the offer buffer is part of the handle's workspace. */
int knng_propagate_pairwise(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                            int32_t k, int32_t rounds, const int32_t* ids_in, const float* dists_in, int32_t* ids,
                            float* dists, void* stream);

/* Divisions used by the last build on h (p->T unless p->r_stop > 0) and, for
 * an adaptive build, their effective rates r_1.. (Sec. 3.2: the share of
 * list entries after division m that were not there after division m - 1;
 * r_1 = 1), up to cap of them written to the host array rates.  Valid after
 * the build's work completed (the adaptive build synchronises its stream). */
int knng_divisions_used(const knng_handle* h, int32_t* m, float* rates, int32_t cap);

/* ---- learned partitioner ----------------------------------------------- */
/* The paper splits along random principal directions (Sec. 3.4) or random
 * projections (appendix after Lemma 1).  As an alternative the library can
 * split along learned features: a network z = tanh(W2 GELU(W1 x + b1) + b2)
 * with z in (-1, 1)^C (C = 16 or 32), where level l < C of tree t splits
 * every node at the median of feature pi_t(l) (pi_t a Philox permutation of
 * the features, a function of (seed, t)) -- unless that feature has become
 * flat inside the node (range within the node below 2% of its range over all
 * points), in which case, as on deeper levels, the node splits along its
 * random direction.  The network
 * is trained on edges of k-NN graphs built by the method itself, so that
 * neighbours stay on the same side of those medians and fewer trees reach
 * the same recall.  Parameters are FP32 (packed W1[H][d] | b1[H] | W2[C][H] |
 * b2[C]); inference is BF16 on the tensor cores (d <= 128). */
typedef struct knng_mlp knng_mlp;

/* A network d_in -> hidden -> d_out on `device`, weights N(0, 1/fan_in)
 * from `seed`, biases 0.  d_in 1..1024, hidden 16..256 (multiple of 16),
 * d_out 16 or 32. */
int knng_mlp_create(int32_t device, int32_t d_in, int32_t hidden, int32_t d_out, uint64_t seed, knng_mlp** out);
int knng_mlp_destroy(knng_mlp* m);
int knng_mlp_param_count(const knng_mlp* m, int64_t* count);
/* Copies the packed parameters to / from HOST memory. */
int knng_mlp_get_params(const knng_mlp* m, float* host);
int knng_mlp_set_params(knng_mlp* m, const float* host);
/* Loss and packed gradient (device, param_count floats) of one batch of B
 * edges: Xpairs is device FP32 [2B][d_in], rows b and B+b the two endpoints
 * of edge b.  *loss is written on the host; synchronises `stream`. */
int knng_mlp_loss_grad(knng_mlp* m, const float* Xpairs, int32_t B, float* loss, float* grad, void* stream);
/* `steps` Adam steps (lr, betas 0.9/0.999) on batches of batch_edges edges
 * drawn (Philox, from `seed`) from the graph ids[n][k] over X (device).
 * *last_loss (host, may be NULL) gets the loss of the last step. */
int knng_mlp_train(knng_mlp* m, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, const int32_t* ids,
                   int32_t k, int32_t steps, int32_t batch_edges, float lr, uint64_t seed, float* last_loss,
                   void* stream);
/* Binary file with a header and the packed FP32 parameters. */
int knng_mlp_save(const knng_mlp* m, const char* path);
int knng_mlp_load(knng_mlp* m, const char* path);
/* Adam state of the training loop (to resume training where it stopped):
 * the first and second moment estimates (HOST, param_count floats each) and
 * the number of steps taken, which sets the bias corrections 1 - 0.9^t and
 * 1 - 0.999^t of the next step.  A new network starts at zero moments and
 * t = 0.  set_adam_state rejects t < 0 with KNNG_ERR_INVALID_ARG. */
int knng_mlp_get_adam_state(const knng_mlp* m, float* m1_host, float* m2_host, int64_t* t);
int knng_mlp_set_adam_state(knng_mlp* m, const float* m1_host, const float* m2_host, int64_t t);
/* Features of every point: Z (device, FP32 [n][d_out]), BF16 inference. */
int knng_mlp_forward(knng_handle* h, knng_mlp* m, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                     float* Z, void* stream);
/* knng_build with learned splits (the network's d_in must equal d).
 * p->partitioner selects how the network's outputs z (d_out per point,
 * BF16 inference) split the points: KNNG_PART_RANDOM -- the random
 * partition trees of knng_build on the points z (a random direction per
 * node in the learned space, median split); KNNG_PART_PCA -- principal-
 * direction trees on z; KNNG_PART_FEATURES -- level l < d_out of tree t
 * splits at the median of one output (a per-tree Philox permutation of the
 * outputs), while that output still varies inside the node, and random
 * directions in the input space elsewhere; KNNG_PART_FEATURES_PCA -- the
 * same with principal directions of the input (knng_partition_pca) in place
 * of the random ones.  Leaf graphs, merge and propagation use X. */
int knng_build_learned(knng_handle* h, knng_mlp* m, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                       const knng_params* p, int32_t* ids, float* dists, void* stream);
/* The partition stage of knng_build_learned with KNNG_PART_FEATURES: the T
 * canonical leaf sets (perm, device [T][n], as knng_partition writes them)
 * of the per-level learned-feature splits.  Level l < d_out of tree t splits
 * every node at the median of output f = pi_t(l) (key ord(z_f) << 32 | id)
 * when the node's range of z_f, max - min in FP32, exceeds 0.02 x (the
 * range of z_f over all points), FP32 product; otherwise, and on levels
 * l >= d_out, at the median of the node's random direction (as
 * knng_partition).  pi_t: Fisher-Yates over 0..d_out-1, i = d_out-1 down to
 * 1, j = w.x mod (i + 1) with w = Philox4x32-10(counter (t, 0x4C524E44, i,
 * 0), key seed).  Z (device, may be NULL) receives the network outputs used,
 * FP32 [n][d_out].  T <= 32, d <= 128. */
int knng_partition_learned(knng_handle* h, knng_mlp* m, const void* X, int32_t dtype, int64_t n, int32_t d,
                           int64_t ld, int32_t T, int32_t g, uint64_t seed, int32_t* perm, float* Z,
                           void* stream);

/* ---- propagation without device allocation ---------------------------- */
/* The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory on their call path -- for example a plugin
 * inside an application whose memory manager already owns all device memory,
 * or a latency-critical loop that cannot pay for the implicit synchronisation
 * of cudaMalloc/cudaFree.  It computes exactly what knng_propagate computes
 * (same kernel, same results), needs no handle, and never allocates: the
 * lists between rounds live in one fixed 16 MiB device array that the library
 * reserves when it is loaded, held by every GPU that loads the library until
 * the process exits.
 *  - Runs on the CURRENT device; X, ids_in, dists_in, ids, dists are device
 *    pointers there, with the layouts of knng_propagate.
 *  - Limits: n <= 524288 and n*k <= 524288; larger requests return
 *    KNNG_ERR_LIMIT without doing any work.  Other bad arguments return
 *    KNNG_ERR_INVALID_ARG; a failed launch returns KNNG_ERR_CUDA.
 *  - The first call on a device looks up the array's device address (once
 *    per device) and keeps it for the life of the process; make that first
 *    call before any stream capture.  A device reset (cudaDeviceReset, or a
 *    primary-context reset by another library) may move the array: after
 *    one, restart the process before calling again.
 *  - dtype F32, F16 or U8, with the alignment rule of knng_propagate.
 *  - Every call shares the one array, which keeps the previous call's
 *    contents (nothing in it needs to start at zero): calls whose work
 *    overlaps on the GPU -- on different streams, or from different host
 *    threads -- race on it and must be serialised by the caller. */
int knng_propagate_noalloc(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, int32_t k,
                           int32_t rounds, const int32_t* ids_in, const float* dists_in, int32_t* ids,
                           float* dists, void* stream);

/* ---- measurement ----------------------------------------------------- */
/* Scales every row of X[n][d] to unit length in FP32 and writes it to the
 * device array Xn (rows of ldn >= d floats; entries d..ldn-1 set to 0): the
 * squared norm is summed in the canonical order of the projection (lane
 * partials over j = 128c + 4l + e, pairwise rounds 16, 8, 4, 2, 1), then
 * sqrtf and one division per entry (IEEE).  A zero row stays zero.  This is
 * the first step of KNNG_METRIC_COSINE. */
int knng_normalize_rows(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, float* Xn,
                        int64_t ldn, void* stream);

/* Exact k-NN lists (Def. 1) of nq query points against all n points, by
 * brute force with the same FP32 distance as the graph (the yardstick of the
 * accuracy measure of Sec. 4).  queries: device int32 [nq] point ids;
 * ids, dists: device [nq][k], ordered by (distance, id). */
int knng_exact_knn(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                   const int32_t* queries, int64_t nq, int32_t k, int32_t* ids, float* dists,
                   void* stream);

/* Stage timing.  With events set (nevents >= 4 + prop_rounds, each a
 * cudaEvent_t created by the caller), knng_build records events[0] before
 * the divisions, [1] after them, [2] after the leaf graphs, [3] after the
 * merge and [4 + r] after propagation round r, all on the build's stream.
 * Pass NULL / 0 to stop recording. */
int knng_set_stage_events(knng_handle* h, void* const* events, int32_t nevents);

/* Number of CUDA kernels the library has launched in this process so far
 * (all handles); a diagnostic for counting launches per build. */
int knng_launch_counter(uint64_t* count);

#ifdef __cplusplus
}
#endif

#endif /* KNNG_H */
