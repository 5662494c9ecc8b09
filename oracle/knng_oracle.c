/*
 * CPU oracle for the k-NN graph construction of Wang, Wang, Zeng, Tu, Gan and
 * Li, "Scalable k-NN graph construction" (arXiv:1307.7852).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  It is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no source
 * with the CUDA library and includes none of its headers.
 *
 * Arithmetic: distances in FP64 (reported rounded to FP32).  The projection
 * used to split a node is the one FP32 quantity that must match the GPU bit
 * for bit, so it is written out in the fixed summation order that defines it
 * (see orc_project).  Compile with -ffp-contract=off so that the compiler
 * fuses nothing that is not written as fmaf.
 *
 * Where the paper is silent, the readings below are used (the CUDA library
 * follows the same ones):
 *   - rho is the squared Euclidean distance (ranks like the Euclidean
 *     distance of Def. 1; the square root is not taken).
 *   - Ties are broken by point id: lists are ordered by (D, id) ascending.
 *   - Random directions (App., after the proof of Lemma 1, which draws the
 *     projection vector a at random) use Philox4x32-10 and a triangular law
 *     on multiples of 2^-16 instead of a Gaussian, so that host and device
 *     agree bit for bit without transcendental functions.
 *   - A node is split at the median of the projections (App., after Lemma 1)
 *     into the floor(m/2) smallest keys (left child 2v) and the rest (right
 *     child 2v+1); the key is (ord(s) << 32 | id).  A node with m <= g is a
 *     leaf (Sec. 3.1 stops at "smaller than g"; the leaf-size bound used here
 *     is "at most g").
 *   - Propagation (Sec. 3.2) is the first-order form analysed in Theorem 1:
 *     one synchronous round replaces every list by the k best of its own
 *     members and its neighbours' members.  The best-first form with a visit
 *     budget (Sec. 3.2) and pairwise updating (Sec. 3.4) are synchronous
 *     passes too (orc_propagate_best_first, orc_propagate_pairwise).
 *   - The cosine distance is 1 - cos, computed as |u - v|^2 / 2 between the
 *     rows scaled to unit length in FP32 (orc_normalize_rows).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror and Shaw, "Parallel random numbers:   */
/* as easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 Philox S-box with the */
/* published multipliers and Weyl key increments.                           */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Random direction of node v at level `level` of tree t (App., after the    */
/* proof of Lemma 1: the projection vector a is drawn at random; one vector  */
/* per node as in a random projection tree).  Entry j takes word j mod 4 of  */
/* Philox(key = seed, counter = (t, level, v, j / 4)) and maps the 32-bit    */
/* word u to ((u & 0xFFFF) + (u >> 16) - 65535) / 65536, a triangular value  */
/* in (-1, 1) that FP32 holds exactly.                                       */
/* ------------------------------------------------------------------------ */
void orc_direction(uint64_t seed, uint32_t t, uint32_t level, uint32_t v, int d, float* a)
{
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    for (int j = 0; j < d; ++j) {
        uint32_t ctr[4] = {t, level, v, (uint32_t)(j / 4)};
        uint32_t word[4];
        orc_philox4x32_10(ctr, key, word);
        uint32_t u = word[j % 4];
        int32_t num = (int32_t)(u & 0xFFFFu) + (int32_t)(u >> 16) - 65535;
        a[j] = (float)num / 65536.0f; /* exact: |num| < 2^17 */
    }
}

/* ------------------------------------------------------------------------ */
/* Projection s = a^T x in FP32, in the fixed order that defines it:         */
/* 32 partial sums ("lanes"); lane l takes the entries j = 128c + 4l + e for */
/* chunk c = 0, 1, ... and e = 0..3 (j < d), each as s_l = fmaf(x_j, a_j,    */
/* s_l) starting from +0; then five pairwise rounds s_l <- s_l + s_(l xor o) */
/* for o = 16, 8, 4, 2, 1.  The value of lane 0 is the projection.          */
/* ------------------------------------------------------------------------ */
float orc_project(const float* x, const float* a, int d)
{
    float s[32];
    for (int l = 0; l < 32; ++l) s[l] = 0.0f;
    int nchunks = (d + 127) / 128;
    for (int l = 0; l < 32; ++l)
        for (int c = 0; c < nchunks; ++c)
            for (int e = 0; e < 4; ++e) {
                int j = 128 * c + 4 * l + e;
                if (j < d) s[l] = fmaf(x[j], a[j], s[l]);
            }
    for (int o = 16; o >= 1; o >>= 1) {
        float nxt[32];
        for (int l = 0; l < 32; ++l) nxt[l] = s[l] + s[l ^ o];
        for (int l = 0; l < 32; ++l) s[l] = nxt[l];
    }
    return s[0];
}

/* Order-preserving map of an FP32 value to an unsigned 32-bit integer:      */
/* sign bit clear -> set the sign bit; sign bit set -> invert every bit.     */
uint32_t orc_ord(float f)
{
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

/* ------------------------------------------------------------------------ */
/* Distances and (D, id) ordering.                                          */
/* ------------------------------------------------------------------------ */
static double sqdist64(const float* x, const float* y, int d)
{
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = (double)x[j] - (double)y[j];
        s += t * t;
    }
    return s;
}

static double sqdist64_dd(const double* x, const double* y, int d)
{
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = x[j] - y[j];
        s += t * t;
    }
    return s;
}

typedef struct {
    double D;
    int32_t id;
} cand_t;

static int cmp_cand(const void* pa, const void* pb)
{
    const cand_t* a = (const cand_t*)pa;
    const cand_t* b = (const cand_t*)pb;
    if (a->D < b->D) return -1;
    if (a->D > b->D) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

static int cmp_u64(const void* pa, const void* pb)
{
    uint64_t a = *(const uint64_t*)pa, b = *(const uint64_t*)pb;
    return (a > b) - (a < b);
}

static int cmp_i32(const void* pa, const void* pb)
{
    int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
    return (a > b) - (a < b);
}

/* Sort the candidates by (D, id) and write the first k; pad with id -1 and
 * distance +inf when fewer than k exist. */
static void emit_topk(cand_t* c, int64_t cnt, int k, int32_t* ids, float* dists)
{
    qsort(c, (size_t)cnt, sizeof(cand_t), cmp_cand);
    for (int e = 0; e < k; ++e) {
        if (e < cnt) {
            ids[e] = c[e].id;
            dists[e] = (float)c[e].D;
        } else {
            ids[e] = -1;
            dists[e] = INFINITY;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* One random partition tree (Sec. 3.1): recursive bisection at the median   */
/* of the projections until a subset holds at most g points.  Leaves are     */
/* emitted left to right, each with its member ids sorted ascending; this is */
/* the canonical leaf set.                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    const float* X;
    int d;
    int64_t ld;
    uint64_t seed;
    uint32_t t;
    int g;
    const float* dirs; /* optional: direction of node (level, v) in row 2^level - 1 + v */
    int32_t* perm;     /* output, n entries */
    int64_t* leaf_off; /* output, nleaves + 1 entries */
    int64_t nleaves;
    int64_t pos;
} part_ctx;

static void split_node(part_ctx* c, int32_t* ids, int64_t m, uint32_t level, uint32_t v)
{
    if (m <= c->g) {
        qsort(ids, (size_t)m, sizeof(int32_t), cmp_i32);
        memcpy(c->perm + c->pos, ids, (size_t)m * sizeof(int32_t));
        c->leaf_off[c->nleaves++] = c->pos;
        c->pos += m;
        return;
    }
    float* a = (float*)malloc((size_t)c->d * sizeof(float));
    uint64_t* keys = (uint64_t*)malloc((size_t)m * sizeof(uint64_t));
    if (c->dirs)
        memcpy(a, c->dirs + (((int64_t)1 << level) - 1 + v) * c->d, (size_t)c->d * sizeof(float));
    else
        orc_direction(c->seed, c->t, level, v, c->d, a);
    for (int64_t i = 0; i < m; ++i) {
        float s = orc_project(c->X + (int64_t)ids[i] * c->ld, a, c->d);
        keys[i] = ((uint64_t)orc_ord(s) << 32) | (uint32_t)ids[i];
    }
    qsort(keys, (size_t)m, sizeof(uint64_t), cmp_u64);
    int64_t ml = m / 2;
    int32_t* left = (int32_t*)malloc((size_t)ml * sizeof(int32_t));
    int32_t* right = (int32_t*)malloc((size_t)(m - ml) * sizeof(int32_t));
    for (int64_t i = 0; i < ml; ++i) left[i] = (int32_t)(keys[i] & 0xFFFFFFFFu);
    for (int64_t i = ml; i < m; ++i) right[i - ml] = (int32_t)(keys[i] & 0xFFFFFFFFu);
    free(keys);
    free(a);
    split_node(c, left, ml, level + 1, 2 * v);
    split_node(c, right, m - ml, level + 1, 2 * v + 1);
    free(left);
    free(right);
}

/* Number of leaves of a tree over n points with leaf size g (depends on n, g
 * only: every split halves a node into floor(m/2) and ceil(m/2)). */
static int64_t count_leaves(int64_t m, int g)
{
    if (m <= g) return 1;
    return count_leaves(m / 2, g) + count_leaves(m - m / 2, g);
}

int64_t orc_leaf_count(int64_t n, int g)
{
    return count_leaves(n, g);
}

/* perm: n entries; leaf_off: orc_leaf_count(n, g) + 1 entries. */
int orc_partition(const float* X, int64_t n, int d, int64_t ld, uint64_t seed, uint32_t t, int g,
                  int32_t* perm, int64_t* leaf_off)
{
    part_ctx c;
    c.X = X;
    c.d = d;
    c.ld = ld;
    c.seed = seed;
    c.t = t;
    c.g = g;
    c.perm = perm;
    c.leaf_off = leaf_off;
    c.nleaves = 0;
    c.pos = 0;
    c.dirs = NULL;
    int32_t* ids = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) ids[i] = (int32_t)i;
    split_node(&c, ids, n, 0, 0);
    free(ids);
    leaf_off[c.nleaves] = n;
    return 0;
}

/* The same tree with given split directions instead of the random ones:
 * dirs holds the direction of node (level, v) in row 2^level - 1 + v (rows of
 * d floats).  Used to replay a partition whose directions were computed
 * elsewhere (the principal directions of Sec. 3.4). */
int orc_partition_dirs(const float* X, int64_t n, int d, int64_t ld, const float* dirs, int g, int32_t* perm,
                       int64_t* leaf_off)
{
    part_ctx c;
    c.X = X;
    c.d = d;
    c.ld = ld;
    c.seed = 0;
    c.t = 0;
    c.g = g;
    c.perm = perm;
    c.leaf_off = leaf_off;
    c.nleaves = 0;
    c.pos = 0;
    c.dirs = dirs;
    int32_t* ids = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) ids[i] = (int32_t)i;
    split_node(&c, ids, n, 0, 0);
    free(ids);
    leaf_off[c.nleaves] = n;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Learned-feature splits (not in the paper; the learned partitioner's       */
/* per-level feature mode).  Z holds C network outputs per point (FP32, row  */
/* i at Z + i*C).  Tree t uses the feature order pi_t, a Fisher-Yates         */
/* shuffle of 0..C-1 driven by Philox4x32-10: for i = C-1 down to 1, word 0  */
/* of Philox(counter (t, 0x4C524E44, i, 0), key seed) modulo i+1 is the      */
/* index j swapped with i.  A node at level l < C splits at the median of    */
/* feature f = pi_t(l) (key ord(z_f) << 32 | id) when its range inside the   */
/* node exceeds tau times its range over all points -- both ranges are       */
/* max - min in FP32 and the product is rounded to FP32 -- and otherwise,    */
/* like every node at level >= C, at the median of its random direction.    */
/* ------------------------------------------------------------------------ */
void orc_feature_order(uint64_t seed, uint32_t t, int C, int32_t* order)
{
    const uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    for (int c = 0; c < C; ++c) order[c] = c;
    for (int i = C - 1; i > 0; --i) {
        const uint32_t ctr[4] = {t, 0x4C524E44u, (uint32_t)i, 0u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        const int j = (int)(w[0] % (uint32_t)(i + 1));
        const int32_t tmp = order[i];
        order[i] = order[j];
        order[j] = tmp;
    }
}

typedef struct {
    part_ctx base;
    const float* Z;
    int C;
    const int32_t* order;
    const float* zrange; /* range of every feature over all points */
    float tau;
} feat_ctx;

static void split_node_feat(feat_ctx* f, int32_t* ids, int64_t m, uint32_t level, uint32_t v)
{
    part_ctx* c = &f->base;
    if (m <= c->g) {
        qsort(ids, (size_t)m, sizeof(int32_t), cmp_i32);
        memcpy(c->perm + c->pos, ids, (size_t)m * sizeof(int32_t));
        c->leaf_off[c->nleaves++] = c->pos;
        c->pos += m;
        return;
    }
    uint64_t* keys = (uint64_t*)malloc((size_t)m * sizeof(uint64_t));
    int learned = 0;
    int feat = 0;
    if ((int)level < f->C) {
        feat = f->order[level];
        float lo = f->Z[(int64_t)ids[0] * f->C + feat], hi = lo;
        for (int64_t i = 1; i < m; ++i) {
            const float z = f->Z[(int64_t)ids[i] * f->C + feat];
            if (z < lo) lo = z;
            if (z > hi) hi = z;
        }
        const float span = hi - lo;
        const float bar = f->tau * f->zrange[feat];
        learned = span > bar;
    }
    if (learned) {
        for (int64_t i = 0; i < m; ++i)
            keys[i] = ((uint64_t)orc_ord(f->Z[(int64_t)ids[i] * f->C + feat]) << 32) | (uint32_t)ids[i];
    } else {
        float* a = (float*)malloc((size_t)c->d * sizeof(float));
        orc_direction(c->seed, c->t, level, v, c->d, a);
        for (int64_t i = 0; i < m; ++i) {
            const float s = orc_project(c->X + (int64_t)ids[i] * c->ld, a, c->d);
            keys[i] = ((uint64_t)orc_ord(s) << 32) | (uint32_t)ids[i];
        }
        free(a);
    }
    qsort(keys, (size_t)m, sizeof(uint64_t), cmp_u64);
    const int64_t ml = m / 2;
    int32_t* left = (int32_t*)malloc((size_t)ml * sizeof(int32_t));
    int32_t* right = (int32_t*)malloc((size_t)(m - ml) * sizeof(int32_t));
    for (int64_t i = 0; i < ml; ++i) left[i] = (int32_t)(keys[i] & 0xFFFFFFFFu);
    for (int64_t i = ml; i < m; ++i) right[i - ml] = (int32_t)(keys[i] & 0xFFFFFFFFu);
    free(keys);
    split_node_feat(f, left, ml, level + 1, 2 * v);
    split_node_feat(f, right, m - ml, level + 1, 2 * v + 1);
    free(left);
    free(right);
}

/* Canonical leaf set of tree t under learned-feature splits (perm: n
 * entries; leaf_off: orc_leaf_count(n, g) + 1 entries). */
int orc_partition_features(const float* X, int64_t n, int d, int64_t ld, const float* Z, int C, uint64_t seed,
                           uint32_t t, int g, float tau, int32_t* perm, int64_t* leaf_off)
{
    if (C < 1 || C > 64) return -1;
    int32_t order[64];
    orc_feature_order(seed, t, C, order);
    float zrange[64];
    for (int c = 0; c < C; ++c) {
        float lo = Z[c], hi = Z[c];
        for (int64_t i = 1; i < n; ++i) {
            const float z = Z[i * C + c];
            if (z < lo) lo = z;
            if (z > hi) hi = z;
        }
        zrange[c] = hi - lo;
    }
    feat_ctx f;
    f.base.X = X;
    f.base.d = d;
    f.base.ld = ld;
    f.base.seed = seed;
    f.base.t = t;
    f.base.g = g;
    f.base.perm = perm;
    f.base.leaf_off = leaf_off;
    f.base.nleaves = 0;
    f.base.pos = 0;
    f.base.dirs = NULL;
    f.Z = Z;
    f.C = C;
    f.order = order;
    f.zrange = zrange;
    f.tau = tau;
    int32_t* ids = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    for (int64_t i = 0; i < n; ++i) ids[i] = (int32_t)i;
    split_node_feat(&f, ids, n, 0, 0);
    free(ids);
    leaf_off[f.base.nleaves] = n;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Leaf graph (Sec. 3.1): brute force inside each subset.  For every point i */
/* of a leaf, the k nearest other members by (D, id).  ids/dists: [n, k],    */
/* row i belongs to point i.                                                 */
/* ------------------------------------------------------------------------ */
int orc_leaf_knn(const float* X, int64_t n, int d, int64_t ld, const int32_t* perm,
                 const int64_t* leaf_off, int64_t nleaves, int k, int32_t* ids, float* dists)
{
    (void)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t L = 0; L < nleaves; ++L) {
        int64_t b = leaf_off[L], e = leaf_off[L + 1];
        cand_t* c = (cand_t*)malloc((size_t)(e - b) * sizeof(cand_t));
        for (int64_t a = b; a < e; ++a) {
            int32_t i = perm[a];
            int64_t cnt = 0;
            for (int64_t q = b; q < e; ++q) {
                int32_t j = perm[q];
                if (j == i) continue;
                c[cnt].D = sqdist64(X + (int64_t)i * ld, X + (int64_t)j * ld, d);
                c[cnt].id = j;
                ++cnt;
            }
            emit_topk(c, cnt, k, ids + (int64_t)i * k, dists + (int64_t)i * k);
        }
        free(c);
    }
    return 0;
}

/* Leaf graph through a reduced-precision candidate stage: for every point i
 * of a leaf, the kp nearest other members by (Dq, id), where Dq is the FP64
 * squared distance between the quantised-and-dequantised rows Xq (n x d,
 * row-major), then the k nearest of those kp by the exact (D, id). */
int orc_leaf_knn_quant(const float* X, int64_t n, int d, int64_t ld, const double* Xq,
                       const int32_t* perm, const int64_t* leaf_off, int64_t nleaves, int k,
                       int kp, int32_t* ids, float* dists)
{
    (void)n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t L = 0; L < nleaves; ++L) {
        int64_t b = leaf_off[L], e = leaf_off[L + 1];
        cand_t* c = (cand_t*)malloc((size_t)(e - b) * sizeof(cand_t));
        for (int64_t a = b; a < e; ++a) {
            int32_t i = perm[a];
            int64_t cnt = 0;
            for (int64_t q = b; q < e; ++q) {
                int32_t j = perm[q];
                if (j == i) continue;
                c[cnt].D = sqdist64_dd(Xq + (int64_t)i * d, Xq + (int64_t)j * d, d);
                c[cnt].id = j;
                ++cnt;
            }
            qsort(c, (size_t)cnt, sizeof(cand_t), cmp_cand);
            int64_t keep = cnt < kp ? cnt : kp;
            for (int64_t r = 0; r < keep; ++r)
                c[r].D = sqdist64(X + (int64_t)i * ld, X + (int64_t)c[r].id * ld, d);
            emit_topk(c, keep, k, ids + (int64_t)i * k, dists + (int64_t)i * k);
        }
        free(c);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Combination of the T base graphs (Sec. 3.1): unite the adjacency lists of */
/* every point and keep its k nearest.  lists: [T, n, k] ids (-1 = empty).   */
/* Distances are recomputed from X, so duplicates collapse by id.           */
/* ------------------------------------------------------------------------ */
int orc_merge(const float* X, int64_t n, int d, int64_t ld, int T, int k, const int32_t* lists,
              int32_t* ids, float* dists)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < n; ++p) {
        int32_t* u = (int32_t*)malloc((size_t)T * k * sizeof(int32_t));
        int64_t cnt = 0;
        for (int t = 0; t < T; ++t)
            for (int e = 0; e < k; ++e) {
                int32_t q = lists[((int64_t)t * n + p) * k + e];
                if (q < 0 || q == p) continue;
                u[cnt++] = q;
            }
        qsort(u, (size_t)cnt, sizeof(int32_t), cmp_i32);
        cand_t* c = (cand_t*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(cand_t));
        int64_t m = 0;
        for (int64_t e = 0; e < cnt; ++e) {
            if (e > 0 && u[e] == u[e - 1]) continue;
            c[m].id = u[e];
            c[m].D = sqdist64(X + p * ld, X + (int64_t)u[e] * ld, d);
            ++m;
        }
        emit_topk(c, m, k, ids + p * k, dists + p * k);
        free(c);
        free(u);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One round of first-order neighbourhood propagation (Sec. 3.2, Theorem 1): */
/* the candidates of p are its current neighbours and their neighbours,     */
/* without p; the new list is the k best candidates by (D, id).  All lists   */
/* are read from the input graph (a synchronous round).                     */
/* ------------------------------------------------------------------------ */
/* First-order candidates of p (its list and its neighbours' lists, without
 * p, deduplicated) and the k best of them by (D, id). */
static void propagate_point(const float* X, int64_t n, int d, int64_t ld, int k, const int32_t* in_ids,
                            int64_t p, int32_t* ids, float* dists)
{
    int64_t cap = (int64_t)k + (int64_t)k * k;
    int32_t* u = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    int64_t cnt = 0;
    for (int e = 0; e < k; ++e) {
        int32_t q = in_ids[p * k + e];
        if (q < 0) continue;
        if (q != p) u[cnt++] = q;
        for (int f = 0; f < k; ++f) {
            int32_t o = in_ids[(int64_t)q * k + f];
            if (o < 0 || o == p) continue;
            u[cnt++] = o;
        }
    }
    qsort(u, (size_t)cnt, sizeof(int32_t), cmp_i32);
    cand_t* c = (cand_t*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(cand_t));
    int64_t m = 0;
    for (int64_t e = 0; e < cnt; ++e) {
        if (e > 0 && u[e] == u[e - 1]) continue;
        c[m].id = u[e];
        c[m].D = sqdist64(X + p * ld, X + (int64_t)u[e] * ld, d);
        ++m;
    }
    emit_topk(c, m, k, ids, dists);
    free(c);
    free(u);
    (void)n;
}

int orc_propagate(const float* X, int64_t n, int d, int64_t ld, int k, const int32_t* in_ids,
                  int32_t* ids, float* dists)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < n; ++p) propagate_point(X, n, d, ld, k, in_ids, p, ids + p * k, dists + p * k);
    return 0;
}

/* The same round for the points rows[0 .. nrows) only: row r of ids/dists
 * ([nrows][k]) is the new list of point rows[r]. */
int orc_propagate_rows(const float* X, int64_t n, int d, int64_t ld, int k, const int32_t* in_ids,
                       const int32_t* rows, int64_t nrows, int32_t* ids, float* dists)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nrows; ++r)
        propagate_point(X, n, d, ld, k, in_ids, rows[r], ids + r * k, dists + r * k);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Canonical FP32 squared distance (a reading: the paper fixes no FP32      */
/* arithmetic).  The entries are cut into blocks of 32, b = 0, 1, ...; in   */
/* block b, partial q (0..7) sums s_q = fmaf(t_j, t_j, s_q) over            */
/* j = 32b + 4q + e, e = 0..3 (entries past d contribute nothing), with     */
/* t_j = x_j - y_j; the block's value is                                    */
/*     B_b = ((s_0 + s_4) + (s_2 + s_6)) + ((s_1 + s_5) + (s_3 + s_7)),     */
/* and the distance is B_0 + B_1 + B_2 + ... added in block order.  Every   */
/* term is non-negative, so the relative error is at most                   */
/* (4 + 3 + ceil(d/32) + 1) units of 2^-24 (the last for the difference):   */
/* 2.3e-6 at d = 960, 8.1e-6 at d = 4096.  It is symmetric in x and y and   */
/* exact on integer rows whose squared distances stay below 2^24.  Used     */
/* where an FP32 distance decides an order (the best-first queue below),    */
/* so that the decision is the kernel's.                                    */
/* ------------------------------------------------------------------------ */
float orc_canon_dist32(const float* x, const float* y, int d)
{
    const int nblocks = (d + 31) / 32;
    float total = 0.0f;
    for (int b = 0; b < nblocks; ++b) {
        float s[8];
        for (int q = 0; q < 8; ++q) {
            s[q] = 0.0f;
            for (int e = 0; e < 4; ++e) {
                const int j = 32 * b + 4 * q + e;
                if (j < d) {
                    const float t = x[j] - y[j];
                    s[q] = fmaf(t, t, s[q]);
                }
            }
        }
        const float blk = ((s[0] + s[4]) + (s[2] + s[6])) + ((s[1] + s[5]) + (s[3] + s[7]));
        total = b == 0 ? blk : total + blk;
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Best-first neighbourhood propagation with a visit budget (Sec. 3.2): for  */
/* every point p, over a frozen snapshot of the lists (a synchronous pass):  */
/*   - p's own neighbours are visited first, in list order, and pushed into  */
/*     a priority queue keyed by their distance to p (nearest on top);       */
/*   - then the top point q is popped and its not yet visited neighbours are */
/*     visited, in q's list order, and pushed; and so on,                    */
/*   - until the queue is empty or `budget` points have been visited (the    */
/*     budget may end a list part way);                                      */
/*   - p's new list is the k best of all visited points by (D, id).          */
/* The queue orders by the canonical FP32 distance with ties by id (the      */
/* kernel's decision); the final list by the FP64 distance as elsewhere.     */
/* budget >= k.  Ids outside [0, n) are empty slots.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    float D32;
    int32_t id;
    int popped;
} bf_entry;

static int bf_less(const bf_entry* a, const bf_entry* b)
{
    if (a->D32 != b->D32) return a->D32 < b->D32;
    return a->id < b->id;
}

int orc_propagate_best_first(const float* X, int64_t n, int d, int64_t ld, int k, const int32_t* in_ids, int budget,
                             int32_t* ids, float* dists)
{
    if (budget < k) return -1;
#pragma omp parallel
    {
        int32_t* mark = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        bf_entry* q = (bf_entry*)malloc((size_t)budget * sizeof(bf_entry));
        cand_t* c = (cand_t*)malloc((size_t)budget * sizeof(cand_t));
        for (int64_t i = 0; i < n; ++i) mark[i] = -1;
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = 0; p < n; ++p) {
            const float* xp = X + p * ld;
            int cnt = 0;
            mark[p] = (int32_t)p;
            /* visit o (if new and the budget allows); returns 0 when full */
#define BF_VISIT(o)                                                                   \
    do {                                                                              \
        int32_t o_ = (o);                                                             \
        if (o_ >= 0 && o_ < n && mark[o_] != (int32_t)p) {                            \
            mark[o_] = (int32_t)p;                                                    \
            q[cnt].D32 = orc_canon_dist32(xp, X + (int64_t)o_ * ld, d);               \
            q[cnt].id = o_;                                                           \
            q[cnt].popped = 0;                                                        \
            ++cnt;                                                                    \
        }                                                                             \
    } while (0)
            for (int e = 0; e < k && cnt < budget; ++e) BF_VISIT(in_ids[p * k + e]);
            while (cnt < budget) {
                int top = -1;
                for (int i = 0; i < cnt; ++i)
                    if (!q[i].popped && (top < 0 || bf_less(&q[i], &q[top]))) top = i;
                if (top < 0) break; /* queue empty */
                q[top].popped = 1;
                const int32_t u = q[top].id;
                for (int f = 0; f < k && cnt < budget; ++f) BF_VISIT(in_ids[(int64_t)u * k + f]);
            }
#undef BF_VISIT
            for (int i = 0; i < cnt; ++i) {
                c[i].id = q[i].id;
                c[i].D = sqdist64(xp, X + (int64_t)q[i].id * ld, d);
            }
            emit_topk(c, cnt, k, ids + p * k, dists + p * k);
        }
        free(c);
        free(q);
        free(mark);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* First-order propagation with pairwise updating (Sec. 3.4 "Speedup": when  */
/* v is considered for u's list, u is also considered for v's list), in the  */
/* synchronous form: with C(p) = N(p) u N(N(p)) \ {p} the candidates of the  */
/* plain round, p's new list is the k best of C(p) together with every q     */
/* whose candidates contain p, {q : p in C(q)}.                              */
/* ------------------------------------------------------------------------ */
int orc_propagate_pairwise(const float* X, int64_t n, int d, int64_t ld, int k, const int32_t* in_ids,
                           int32_t* ids, float* dists)
{
    const int64_t cap = (int64_t)k + (int64_t)k * k;
    int32_t* C = (int32_t*)malloc((size_t)(n * cap) * sizeof(int32_t));
    int32_t* len = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    /* pass 1: the candidate sets C(p), deduplicated */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < n; ++p) {
        int32_t* u = C + p * cap;
        int64_t cnt = 0;
        for (int e = 0; e < k; ++e) {
            int32_t qq = in_ids[p * k + e];
            if (qq < 0 || qq >= n) continue;
            if (qq != p) u[cnt++] = qq;
            for (int f = 0; f < k; ++f) {
                int32_t o = in_ids[(int64_t)qq * k + f];
                if (o < 0 || o >= n || o == p) continue;
                u[cnt++] = o;
            }
        }
        qsort(u, (size_t)cnt, sizeof(int32_t), cmp_i32);
        int64_t m = 0;
        for (int64_t e = 0; e < cnt; ++e)
            if (e == 0 || u[e] != u[e - 1]) u[m++] = u[e];
        len[p] = (int32_t)m;
    }
    /* reverse offers: rev[c] = {p : c in C(p)} */
    int64_t* roff = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t p = 0; p < n; ++p)
        for (int32_t e = 0; e < len[p]; ++e) roff[C[p * cap + e] + 1]++;
    for (int64_t i = 0; i < n; ++i) roff[i + 1] += roff[i];
    int32_t* rev = (int32_t*)malloc((size_t)(roff[n] > 0 ? roff[n] : 1) * sizeof(int32_t));
    int64_t* fill = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) fill[i] = roff[i];
    for (int64_t p = 0; p < n; ++p)
        for (int32_t e = 0; e < len[p]; ++e) rev[fill[C[p * cap + e]]++] = (int32_t)p;
    /* pass 2: k best of C(p) u rev(p) */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < n; ++p) {
        const int64_t nr = roff[p + 1] - roff[p];
        int32_t* u = (int32_t*)malloc((size_t)(len[p] + nr + 1) * sizeof(int32_t));
        int64_t cnt = 0;
        for (int32_t e = 0; e < len[p]; ++e) u[cnt++] = C[p * cap + e];
        for (int64_t e = 0; e < nr; ++e) u[cnt++] = rev[roff[p] + e];
        qsort(u, (size_t)cnt, sizeof(int32_t), cmp_i32);
        cand_t* c = (cand_t*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(cand_t));
        int64_t m = 0;
        for (int64_t e = 0; e < cnt; ++e) {
            if (e > 0 && u[e] == u[e - 1]) continue;
            c[m].id = u[e];
            c[m].D = sqdist64(X + p * ld, X + (int64_t)u[e] * ld, d);
            ++m;
        }
        emit_topk(c, m, k, ids + p * k, dists + p * k);
        free(c);
        free(u);
    }
    free(fill);
    free(rev);
    free(roff);
    free(len);
    free(C);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact k-NN lists (Def. 1) of the query points against all n points, by    */
/* brute force; the accuracy of Sec. 4 is measured against these.           */
/* ------------------------------------------------------------------------ */
int orc_knn_exact(const float* X, int64_t n, int d, int64_t ld, int k, const int32_t* queries,
                  int64_t nq, int32_t* ids, float* dists)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < nq; ++a) {
        int32_t p = queries[a];
        cand_t* c = (cand_t*)malloc((size_t)n * sizeof(cand_t));
        int64_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == p) continue;
            c[cnt].D = sqdist64(X + (int64_t)p * ld, X + j * ld, d);
            c[cnt].id = (int32_t)j;
            ++cnt;
        }
        emit_topk(c, cnt, k, ids + a * k, dists + a * k);
        free(c);
    }
    return 0;
}

/* FP64 squared distances of given pairs (a helper for tests and recall). */
int orc_pair_dist(const float* X, int d, int64_t ld, const int32_t* a, const int32_t* b,
                  int64_t npairs, double* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < npairs; ++e)
        out[e] = sqdist64(X + (int64_t)a[e] * ld, X + (int64_t)b[e] * ld, d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cosine metric (App., after the proof of Lemma 1: for the cosine distance  */
/* a random projection builds the partition tree).  Every row is scaled to  */
/* unit length in FP32: its squared norm in the fixed order of orc_project  */
/* (the row itself in place of the direction), the IEEE square root, one    */
/* IEEE division per entry.  A zero row stays zero.  The cosine distance of */
/* two rows, 1 - cos, is then |u - v|^2 / 2 over the scaled rows u, v, so   */
/* the method runs unchanged on the scaled rows and halves the distances.   */
/* ------------------------------------------------------------------------ */
int orc_normalize_rows(const float* X, int64_t n, int d, int64_t ld, float* out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const float* x = X + i * ld;
        float* u = out + i * (int64_t)d;
        const float s = orc_project(x, x, d);
        const float r = sqrtf(s);
        for (int j = 0; j < d; ++j) u[j] = s > 0.0f ? x[j] / r : 0.0f;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision encodings of the candidate stage.                      */
/* ------------------------------------------------------------------------ */

/* Round to the nearest value with `sig` significant bits whose exponent is
 * at least emin (below it the spacing stays 2^(emin - sig + 1)), ties to
 * even.  Written from the definition: scale by the spacing, rint (the
 * default rounding mode rounds half to even), scale back. */
static double round_to_grid(double x, int sig, int emin)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int E;
    frexp(x, &E); /* |x| = f * 2^E, f in [0.5, 1): exponent of x is E - 1 */
    int e = E - 1;
    if (e < emin) e = emin;
    double spacing = ldexp(1.0, e - (sig - 1));
    return rint(x / spacing) * spacing;
}

/* bfloat16: 8 significant bits, FP32's exponent range (min normal 2^-126). */
float orc_bf16_round(float x)
{
    double r = round_to_grid((double)x, 8, -126);
    const double maxbf = ldexp(255.0, 120); /* (2 - 2^-7) * 2^127 */
    if (fabs(r) > maxbf) r = copysign(INFINITY, r);
    return (float)r;
}

/* FP8 E4M3 (the "fn" variant without infinities): 4 significant bits, min
 * normal 2^-6, largest finite 448; out-of-range values saturate to +-448. */
float orc_e4m3_round(float x)
{
    double r = round_to_grid((double)x, 4, -6);
    if (r > 448.0) r = 448.0;
    if (r < -448.0) r = -448.0;
    return (float)r;
}

/* Quantise rows for the candidate stage and return them dequantised in
 * FP64.  mode 1: bfloat16 per entry.  mode 2: E4M3 with one FP32 scale per
 * row, s = max_j |x_j| / 448 (s = 1 for an all-zero row), code = E4M3(x/s)
 * with the division done in FP32; value = s * code. */
int orc_quantize_rows(const float* X, int64_t n, int d, int64_t ld, int mode, double* Xq,
                      float* scales)
{
    for (int64_t i = 0; i < n; ++i) {
        const float* x = X + i * ld;
        double* q = Xq + i * d;
        if (mode == 1) {
            for (int j = 0; j < d; ++j) q[j] = (double)orc_bf16_round(x[j]);
            if (scales) scales[i] = 1.0f;
        } else if (mode == 2) {
            float mx = 0.0f;
            for (int j = 0; j < d; ++j) {
                float ax = fabsf(x[j]);
                if (ax > mx) mx = ax;
            }
            float s = (mx > 0.0f) ? mx / 448.0f : 1.0f;
            for (int j = 0; j < d; ++j) {
                float code = orc_e4m3_round(x[j] / s);
                q[j] = (double)s * (double)code;
            }
            if (scales) scales[i] = s;
        } else {
            for (int j = 0; j < d; ++j) q[j] = (double)x[j];
            if (scales) scales[i] = 1.0f;
        }
    }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
