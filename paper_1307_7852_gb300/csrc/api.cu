// C ABI of the library (include/knng.h): argument checks, the handle with its
// workspace and cached tree plan, and the order of the stages.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/knng.h"
#include "knng_internal.h"

namespace knng {
static std::atomic<unsigned long long> g_launches{0};
void note_launches(int count) { g_launches.fetch_add((unsigned long long)count, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}
}  // namespace knng

using namespace knng;

// A recorded batched build (knng_build_batched): the batch it was recorded
// for, its device tables and the instantiated CUDA graph.
struct BatchGroup {
    int dtype = 0, d = 0;
    int64_t n = 0, ld = 0;
    std::vector<int> members;
    TreePlan plan;
    DevPlan dp;
    const BatchSet* dev_sets = nullptr;
};
struct BatchCache {
    std::vector<uint64_t> sig;
    std::vector<BatchGroup> groups;
    char* tables = nullptr;
    size_t tables_size = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int kernels = 0;  // kernel nodes of the graph
};

struct knng_handle {
    int device = 0;
    char* ws = nullptr;
    size_t ws_size = 0;
    TreePlan plan;
    char* plan_dev = nullptr;
    size_t plan_dev_size = 0;
    DevPlan dplan;
    std::vector<cudaEvent_t> stage_ev;
    int* dev_err = nullptr;  // set by kernels whose bounded waits gave up
    BatchCache batch;
    std::map<TcKey, TcTile> tune;  // tile choices found by knng_autotune
    std::string err;
    int div_used = 0;            // divisions used by the last build
    std::vector<float> div_rates;  // their effective rates r_m (adaptive builds)
    char* staging = nullptr;     // device copies of knng_build_host's buffers (grow-only)
    size_t staging_size = 0;
    long long wait_cycles = 0;   // limit of the leaf kernel's pipeline waits (0: about 1 s)
    unsigned long long* prop_stats = nullptr;  // caller's read counters, 2 per round
    int prop_stats_rounds = 0;
};

namespace {

int fail(knng_handle* h, int code, const char* fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

int cuda_fail(knng_handle* h, cudaError_t e, const char* where)
{
    return fail(h, KNNG_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Grows the workspace to at least `bytes` (stream-ordered free/alloc).
int ensure_ws(knng_handle* h, size_t bytes, cudaStream_t st)
{
    if (bytes <= h->ws_size) return KNNG_OK;
    if (h->ws) {
        cudaFreeAsync(h->ws, st);
        h->ws = nullptr;
        h->ws_size = 0;
    }
    size_t want = bytes + (bytes >> 3) + (1 << 20);
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, want, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, KNNG_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    h->ws = static_cast<char*>(p);
    h->ws_size = want;
    return KNNG_OK;
}

// Makes the handle's tree plan describe (n, g) and uploads it.
int ensure_plan(knng_handle* h, int64_t n, int g, cudaStream_t st)
{
    if (h->plan.n == n && h->plan.g == g && h->plan_dev) return KNNG_OK;
    make_tree_plan(n, g, h->plan);
    const TreePlan& P = h->plan;
    const size_t nb = sizeof(SplitNode) * P.nodes.size();
    const size_t cb = sizeof(Chunk) * P.chunks.size();
    const size_t lb = sizeof(int32_t) * P.leaf_off.size();
    const size_t o_c = (nb + 255) & ~(size_t)255;
    const size_t o_l = (o_c + cb + 255) & ~(size_t)255;
    const size_t total = o_l + lb + 256;
    if (total > h->plan_dev_size) {
        if (h->plan_dev) {
            cudaStreamSynchronize(st);
            cudaFree(h->plan_dev);
        }
        h->plan_dev = nullptr;
        h->plan_dev_size = 0;
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->plan.n = -1;
            return fail(h, KNNG_ERR_OOM, "plan table of %zu bytes", total);
        }
        h->plan_dev = static_cast<char*>(p);
        h->plan_dev_size = total;
    } else {
        cudaStreamSynchronize(st);  // the old plan may still be in use
    }
    cudaError_t e = cudaSuccess;
    if (nb) e = cudaMemcpy(h->plan_dev, P.nodes.data(), nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && cb) e = cudaMemcpy(h->plan_dev + o_c, P.chunks.data(), cb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->plan_dev + o_l, P.leaf_off.data(), lb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        h->plan.n = -1;
        return cuda_fail(h, e, "plan upload");
    }
    h->dplan.nodes = reinterpret_cast<const SplitNode*>(h->plan_dev);
    h->dplan.chunks = reinterpret_cast<const Chunk*>(h->plan_dev + o_c);
    h->dplan.leaf_off = reinterpret_cast<const int32_t*>(h->plan_dev + o_l);
    return KNNG_OK;
}

size_t dtype_size(int32_t dtype)
{
    return dtype == KNNG_DTYPE_F16 ? 2 : dtype == KNNG_DTYPE_U8 ? 1 : 4;
}

int check_x(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, XDesc& x)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    if (!X) return fail(h, KNNG_ERR_INVALID_ARG, "X is NULL");
    if (dtype != KNNG_DTYPE_F32 && dtype != KNNG_DTYPE_F16 && dtype != KNNG_DTYPE_U8)
        return fail(h, KNNG_ERR_INVALID_ARG, "dtype %d", dtype);
    if (n < 2 || n >= (int64_t)1 << 31) return fail(h, KNNG_ERR_INVALID_ARG, "n = %lld out of [2, 2^31)", (long long)n);
    if (d < 1 || d > 4096) return fail(h, KNNG_ERR_INVALID_ARG, "d = %d out of [1, 4096]", d);
    if (ld < d || ld >= (int64_t)1 << 31) return fail(h, KNNG_ERR_INVALID_ARG, "ld = %lld out of [d, 2^31)", (long long)ld);
    const size_t es = dtype_size(dtype);
    const size_t align = dtype == KNNG_DTYPE_F16 ? 8 : dtype == KNNG_DTYPE_U8 ? 4 : 16;
    x.X = X;
    x.dtype = dtype;
    x.n = n;
    x.d = d;
    x.ld = ld;
    x.vec = ((uintptr_t)X % align == 0) && ((size_t)ld * es % align == 0);
    return KNNG_OK;
}

int check_tree(knng_handle* h, int32_t T, int32_t g)
{
    if (T < 1 || T > kMaxT) return fail(h, KNNG_ERR_INVALID_ARG, "T = %d out of [1, %d]", T, kMaxT);
    if (g < 2 || g > kMaxLeaf) return fail(h, KNNG_ERR_INVALID_ARG, "leaf_size = %d out of [2, %d]", g, kMaxLeaf);
    return KNNG_OK;
}

int check_k(knng_handle* h, int32_t k, int32_t g)
{
    if (k < 1 || k > kMaxK) return fail(h, KNNG_ERR_INVALID_ARG, "k = %d out of [1, %d]", k, kMaxK);
    if (g >= 0 && k >= g / 2)
        return fail(h, KNNG_ERR_INVALID_ARG, "k = %d must be below leaf_size/2 = %d", k, g / 2);
    return KNNG_OK;
}

// Leaf graphs of all trees.  With ar.base == nullptr only measures the
// scratch the stage needs.
// all_exact (nullable): left nonzero only when every leaf list is the exact
// k best of its leaf (tensor-core path with exact leaves).
int leaf_stage(knng_handle* h, const TreePlan& P, const DevPlan& dp, const XDesc& x, int T, const int32_t* perm,
               int k, int prec, int mult, int32_t* ids, float* dists, Arena& ar, cudaStream_t st,
               int* all_exact = nullptr)
{
    cudaError_t e;
    const int kp = std::min(mult * k, 128);
    if (prec == KNNG_PREC_FP32) {
        if (!ar.base) return KNNG_OK;
        e = all_exact ? cudaMemsetAsync(all_exact, 0, sizeof(int), st) : cudaSuccess;
        if (e == cudaSuccess) e = run_leaf_knn_f32(x, P, dp, T, perm, k, kp, ids, dists, st);
    } else if (prec == KNNG_PREC_BF16 || prec == KNNG_PREC_FP8E4M3) {
        const auto it = h->tune.find(tc_key(P, x.d, prec));
        const TcTile* tile = it == h->tune.end() ? nullptr : &it->second;
        e = (all_exact && ar.base) ? cudaMemsetAsync(all_exact, 0x01, sizeof(int), st) : cudaSuccess;
        if (e == cudaSuccess)
            e = run_leaf_knn_tc(x, P, dp, T, perm, k, kp, prec, ids, dists, h->dev_err, ar, st, tile, all_exact,
                                h->wait_cycles);
    } else {
        return fail(h, KNNG_ERR_INVALID_ARG, "precision %d", prec);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "leaf k-NN");
    return KNNG_OK;
}

int check_params(knng_handle* h, const knng_params* p, int64_t n)
{
    if (!p) return fail(h, KNNG_ERR_INVALID_ARG, "params is NULL");
    int r;
    if ((r = check_tree(h, p->T, p->leaf_size))) return r;
    if ((r = check_k(h, p->k, n > p->leaf_size ? p->leaf_size : -1))) return r;
    if (p->prop_rounds < 0 || p->prop_rounds > 16) return fail(h, KNNG_ERR_INVALID_ARG, "prop_rounds %d", p->prop_rounds);
    if (p->rescore_mult < 1 || p->rescore_mult > 4) return fail(h, KNNG_ERR_INVALID_ARG, "rescore_mult %d", p->rescore_mult);
    if (p->partitioner != KNNG_PART_RANDOM && p->partitioner != KNNG_PART_PCA)
        return fail(h, KNNG_ERR_INVALID_ARG, "partitioner %d", p->partitioner);
    if (p->metric != KNNG_METRIC_L2 && p->metric != KNNG_METRIC_COSINE)
        return fail(h, KNNG_ERR_INVALID_ARG, "metric %d", p->metric);
    if (p->propagation != KNNG_PROP_FIRST_ORDER && p->propagation != KNNG_PROP_BEST_FIRST &&
        p->propagation != KNNG_PROP_PAIRWISE)
        return fail(h, KNNG_ERR_INVALID_ARG, "propagation %d", p->propagation);
    if (p->propagation == KNNG_PROP_BEST_FIRST && (p->budget < p->k || p->budget > 512))
        return fail(h, KNNG_ERR_INVALID_ARG, "budget %d out of [k, 512]", p->budget);
    if (!(p->r_stop >= 0.f && p->r_stop <= 1.f)) return fail(h, KNNG_ERR_INVALID_ARG, "r_stop out of [0, 1]");
    if (p->reserved != 0) return fail(h, KNNG_ERR_INVALID_ARG, "reserved must be 0");
    return KNNG_OK;
}

// The whole method over one point set (or one forest of sets): divisions,
// leaf graphs, merge, propagation rounds.  Carves its buffers from ar; with
// ar.base == nullptr it only measures them.
int build_pipeline(knng_handle* h, const TreePlan& P, const DevPlan& dp, const XDesc& x_in, const knng_params& p,
                   int32_t* ids, float* dists, Arena& a, cudaStream_t st, bool events,
                   const LearnedFeat* lf = nullptr, bool byte_copy = false, const XDesc* xpart = nullptr)
{
    XDesc x = x_in;
    const int64_t n = x.n;
    const int T = p.T, k = p.k, R = p.prop_rounds;
    const size_t nk = (size_t)n * k;
    // perm | leaf lists | propagation buffers | max(partition, leaf scratch)
    int32_t* perm = a.take<int32_t>((size_t)T * n);
    int32_t* li = a.take<int32_t>((size_t)T * nk);
    float* ld_ = a.take<float>((size_t)T * nk);
    int32_t* bi[2];
    float* bd[2];
    unsigned long long* fl[2];
    for (int b = 0; b < 2; ++b) {
        bi[b] = a.take<int32_t>(nk);
        bd[b] = a.take<float>(nk);
        fl[b] = a.take<unsigned long long>(n);
    }
    // cosine metric: the method runs on the rows scaled to unit length
    const bool cosine = p.metric == KNNG_METRIC_COSINE;
    if (cosine) {
        const int64_t ldn = ((int64_t)x.d + 3) & ~(int64_t)3;
        float* xn = a.take<float>((size_t)n * ldn);
        if (a.base) {
            const cudaError_t e = run_normalize_rows(x, xn, ldn, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "normalize rows");
        }
        x = XDesc{xn, KNNG_DTYPE_F32, n, x.d, ldn, true};
    }
    // float rows that hold only bytes: exact byte copy for the gathering kernels
    uint8_t* xb = nullptr;
    int* xb_bad = nullptr;
    const int64_t ldb = ((int64_t)x.d + 15) & ~(int64_t)15;
    if (byte_copy && !cosine && x.dtype == KNNG_DTYPE_F32 && x.d <= 256) {
        xb = a.take<uint8_t>((size_t)n * ldb);
        xb_bad = a.take<int>(1);
    }
    unsigned long long* rate_cnt = a.take<unsigned long long>(2);
    // the merge's tree masks for the first first-order round (T <= 8)
    const bool tmasks = !(p.r_stop > 0.f) && R > 0 && T <= 8 && p.propagation == KNNG_PROP_FIRST_ORDER;
    uint8_t* tmask = tmasks ? a.take<uint8_t>(nk) : nullptr;
    int* all_exact = tmasks ? a.take<int>(1) : nullptr;
    PcaOpt pca;
    pca.on = p.partitioner == KNNG_PART_PCA;
    if (pca.on && x.d > 1024) return fail(h, KNNG_ERR_UNSUPPORTED, "principal directions support d <= 1024");
    const bool adaptive = p.r_stop > 0.f;
    PairScratch pw;
    if (p.propagation == KNNG_PROP_PAIRWISE && R > 0) pairwise_take(a, n, k, pw);
    const size_t fixed = a.off;
    int r;
    if (!a.base) {
        run_partition(xpart ? *xpart : x, P, dp, T, p.seed, nullptr, a, st, lf);
        const size_t part_end = a.off;
        a.off = fixed;
        if ((r = leaf_stage(h, P, dp, x, T, nullptr, k, p.precision, p.rescore_mult, nullptr, nullptr, a, st)))
            return r;
        a.off = std::max(part_end, a.off);
        return KNNG_OK;
    }
    const bool rec = events && (int)h->stage_ev.size() >= 4 + R;
    auto mark = [&](int i) {
        if (rec) cudaEventRecord(h->stage_ev[i], st);
    };
    mark(0);
    h->div_used = T;
    h->div_rates.clear();
    cudaError_t e;
    if (xb) {
        e = cudaMemsetAsync(xb_bad, 0, sizeof(int), st);
        if (e == cudaSuccess) e = run_byte_copy(x, xb, ldb, xb_bad, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "byte copy");
        x.Xb = xb;
        x.ldb = ldb;
        x.xb_bad = xb_bad;
    }
    int cur = 0;  // bi[cur] / bd[cur]: the merged graph when R > 0
    if (!adaptive) {
        e = run_partition(xpart ? *xpart : x, P, dp, T, p.seed, perm, a, st, lf, 0, &pca, h->dev_err);
        if (e != cudaSuccess) return cuda_fail(h, e, "partition");
        mark(1);
        const size_t part_end = a.off;
        a.off = fixed;  // the partition scratch is dead: the leaf stage reuses it
        if ((r = leaf_stage(h, P, dp, x, T, perm, k, p.precision, p.rescore_mult, li, ld_, a, st, all_exact)))
            return r;
        a.off = std::max(part_end, a.off);
        mark(2);
        int32_t* mi = R == 0 ? ids : bi[0];
        float* md = R == 0 ? dists : bd[0];
        e = run_merge(n, T, k, li, ld_, mi, md, st, tmask, all_exact);
        if (e != cudaSuccess) return cuda_fail(h, e, "merge");
        mark(3);
    } else {
        // Sec. 4: divisions are added one by one until the effective rate
        // r_m of the last one falls below r_stop; trees are partitioned and
        // their leaf graphs built two at a time, then merged one at a time
        // with a host check of r_m after each (a tree past the stop is
        // discarded unused).
        constexpr int kChunk = 2;
        bool stop = false;
        for (int t0 = 0; t0 < T && !stop; t0 += kChunk) {
            const int tc = std::min(kChunk, T - t0);
            const size_t base = a.off;
            e = run_partition(xpart ? *xpart : x, P, dp, tc, p.seed, perm + (size_t)t0 * n, a, st, lf, t0, &pca,
                              h->dev_err);
            if (e != cudaSuccess) return cuda_fail(h, e, "partition");
            const size_t part_end = a.off;
            a.off = base;
            if ((r = leaf_stage(h, P, dp, x, tc, perm + (size_t)t0 * n, k, p.precision, p.rescore_mult,
                                li + (size_t)t0 * nk, ld_ + (size_t)t0 * nk, a, st)))
                return r;
            a.off = std::max(part_end, a.off);
            a.off = base;
            for (int j = 0; j < tc && !stop; ++j) {
                const int t = t0 + j;
                float rate = 1.f;
                if (t == 0) {
                    e = run_merge(n, 1, k, li, ld_, bi[0], bd[0], st);
                    cur = 0;
                } else {
                    unsigned long long hc[2] = {0, 0};
                    e = cudaMemsetAsync(rate_cnt, 0, sizeof hc, st);
                    if (e == cudaSuccess)
                        e = run_merge_add(n, k, bi[cur], bd[cur], li + (size_t)t * nk, ld_ + (size_t)t * nk,
                                          bi[cur ^ 1], bd[cur ^ 1], rate_cnt, st);
                    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, rate_cnt, sizeof hc, cudaMemcpyDeviceToHost, st);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                    cur ^= 1;
                    rate = hc[1] ? (float)((double)hc[0] / (double)hc[1]) : 0.f;
                }
                if (e != cudaSuccess) return cuda_fail(h, e, "merge");
                h->div_rates.push_back(rate);
                if (rate < p.r_stop) {
                    h->div_used = t + 1;
                    stop = true;
                }
            }
        }
        if (R == 0) {
            e = cudaMemcpyAsync(ids, bi[cur], nk * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dists, bd[cur], nk * sizeof(float), cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(h, e, "copy");
        }
        mark(1);
        mark(2);
        mark(3);
    }
    // propagation visits points in the leaf order of tree 0: neighbouring
    // points run together, so candidate rows are shared through L2.
    for (int rd = 0; rd < R; ++rd) {
        const int32_t* si = bi[cur];
        const float* sd = bd[cur];
        const unsigned long long* sf = rd == 0 ? nullptr : fl[cur];
        const bool last = rd == R - 1;
        int32_t* oi = last ? ids : bi[cur ^ 1];
        float* od = last ? dists : bd[cur ^ 1];
        unsigned long long* of = last ? nullptr : fl[cur ^ 1];
        if (p.propagation == KNNG_PROP_BEST_FIRST)
            e = run_propagate_best_first(x, k, p.budget, perm, si, oi, od, st);
        else if (p.propagation == KNNG_PROP_PAIRWISE)
            e = run_propagate_pairwise(x, k, perm, si, sd, sf, oi, od, of, pw, h->dev_err, st);
        else
            e = run_propagate(x, k, perm, si, sd, sf, oi, od, of, st, nullptr, rd == 0 ? tmask : nullptr,
                              rd < h->prop_stats_rounds ? h->prop_stats + 2 * rd : nullptr);
        if (e != cudaSuccess) return cuda_fail(h, e, "propagate");
        cur ^= 1;
        mark(4 + rd);
    }
    if (cosine) {
        // |u - v|^2 / 2 = 1 - cos between unit rows (exact halving)
        e = run_scale(dists, (int64_t)nk, 0.5f, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cosine distances");
    }
    return KNNG_OK;
}

}  // namespace

// ===========================================================================
extern "C" {

const char* knng_status_string(int32_t s)
{
    switch (s) {
        case KNNG_OK: return "ok";
        case KNNG_ERR_INVALID_ARG: return "invalid argument";
        case KNNG_ERR_UNSUPPORTED: return "unsupported";
        case KNNG_ERR_OOM: return "out of device memory";
        case KNNG_ERR_CUDA: return "CUDA error";
        case KNNG_ERR_TIMEOUT: return "device wait timed out";
        case KNNG_ERR_INTERNAL: return "internal error";
        case KNNG_ERR_LIMIT: return "request exceeds a fixed capacity of the library";
        default: return "unknown status";
    }
}

int knng_create(knng_handle** out, int32_t device)
{
    if (!out) return KNNG_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return KNNG_ERR_INVALID_ARG;
    }
    knng_handle* h = new (std::nothrow) knng_handle();
    if (!h) return KNNG_ERR_INTERNAL;
    h->device = device;
    {
        DeviceGuard g(device);
        void* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess || cudaMemset(p, 0, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            if (p) cudaFree(p);
            delete h;
            return KNNG_ERR_OOM;
        }
        h->dev_err = static_cast<int*>(p);
    }
    *out = h;
    return KNNG_OK;
}

int knng_destroy(knng_handle* h)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    {
        DeviceGuard g(h->device);
        cudaDeviceSynchronize();
        if (h->ws) cudaFree(h->ws);
        if (h->plan_dev) cudaFree(h->plan_dev);
        if (h->dev_err) cudaFree(h->dev_err);
        if (h->staging) cudaFree(h->staging);
        BatchCache& B = h->batch;
        if (B.exec) cudaGraphExecDestroy(B.exec);
        if (B.graph) cudaGraphDestroy(B.graph);
        if (B.tables) cudaFree(B.tables);
        if (B.cap) cudaStreamDestroy(B.cap);
        if (B.ev_in) cudaEventDestroy(B.ev_in);
        if (B.ev_out) cudaEventDestroy(B.ev_out);
    }
    delete h;
    return KNNG_OK;
}

const char* knng_last_error(const knng_handle* h)
{
    return h ? h->err.c_str() : "";
}

int knng_leaf_count(int64_t n, int32_t g, int64_t* nleaves)
{
    if (!nleaves || n < 1 || g < 1) return KNNG_ERR_INVALID_ARG;
    TreePlan P;
    make_tree_plan(n, g, P);
    *nleaves = (int64_t)P.leaf_off.size() - 1;
    return KNNG_OK;
}

int knng_leaf_offsets(int64_t n, int32_t g, int64_t* leaf_off)
{
    if (!leaf_off || n < 1 || g < 1) return KNNG_ERR_INVALID_ARG;
    TreePlan P;
    make_tree_plan(n, g, P);
    for (size_t i = 0; i < P.leaf_off.size(); ++i) leaf_off[i] = P.leaf_off[i];
    return KNNG_OK;
}

int knng_partition(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                   int32_t T, int32_t g, uint64_t seed, int32_t* perm, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_tree(h, T, g))) return r;
    if (!perm) return fail(h, KNNG_ERR_INVALID_ARG, "perm is NULL");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = ensure_plan(h, n, g, st))) return r;
    Arena m;
    run_partition(x, h->plan, h->dplan, T, seed, perm, m, st);
    if ((r = ensure_ws(h, m.off, st))) return r;
    Arena a;
    a.base = h->ws;
    cudaError_t e = run_partition(x, h->plan, h->dplan, T, seed, perm, a, st, nullptr, 0, nullptr, h->dev_err);
    if (e != cudaSuccess) return cuda_fail(h, e, "partition");
    return KNNG_OK;
}

int knng_split_levels(int64_t n, int32_t g, int32_t* levels)
{
    if (!levels || n < 1 || g < 1) return KNNG_ERR_INVALID_ARG;
    TreePlan P;
    make_tree_plan(n, g, P);
    *levels = (int32_t)P.levels.size();
    return KNNG_OK;
}

int knng_partition_pca(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, int32_t T,
                       int32_t g, uint64_t seed, int32_t* perm, float* dirs_out, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_tree(h, T, g))) return r;
    if (!perm) return fail(h, KNNG_ERR_INVALID_ARG, "perm is NULL");
    if (d > 1024) return fail(h, KNNG_ERR_UNSUPPORTED, "principal directions support d <= 1024");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = ensure_plan(h, n, g, st))) return r;
    PcaOpt pca;
    pca.on = true;
    pca.out = dirs_out;
    pca.stride = ((((int64_t)1) << h->plan.levels.size()) - 1) * d;
    Arena m;
    run_partition(x, h->plan, h->dplan, T, seed, nullptr, m, st, nullptr, 0, &pca);
    if ((r = ensure_ws(h, m.off, st))) return r;
    Arena a;
    a.base = h->ws;
    const cudaError_t e = run_partition(x, h->plan, h->dplan, T, seed, perm, a, st, nullptr, 0, &pca, h->dev_err);
    if (e != cudaSuccess) return cuda_fail(h, e, "partition");
    return KNNG_OK;
}

int knng_leaf_knn(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                  int32_t T, int32_t g, const int32_t* perm, int32_t k, int32_t precision,
                  int32_t rescore_mult, int32_t* ids, float* dists, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_tree(h, T, g))) return r;
    if ((r = check_k(h, k, n > g ? g : -1))) return r;
    if (!perm || !ids || !dists) return fail(h, KNNG_ERR_INVALID_ARG, "NULL pointer");
    if (rescore_mult < 1 || rescore_mult > 4) return fail(h, KNNG_ERR_INVALID_ARG, "rescore_mult %d", rescore_mult);
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = ensure_plan(h, n, g, st))) return r;
    Arena m;
    if ((r = leaf_stage(h, h->plan, h->dplan, x, T, perm, k, precision, rescore_mult, ids, dists, m, st))) return r;
    if ((r = ensure_ws(h, m.off, st))) return r;
    Arena a;
    a.base = h->ws;
    return leaf_stage(h, h->plan, h->dplan, x, T, perm, k, precision, rescore_mult, ids, dists, a, st);
}

int knng_merge(knng_handle* h, int64_t n, int32_t T, int32_t k, const int32_t* ids_in,
               const float* dists_in, int32_t* ids, float* dists, void* stream)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    if (n < 1 || n >= (int64_t)1 << 31) return fail(h, KNNG_ERR_INVALID_ARG, "n = %lld", (long long)n);
    if (T < 1 || T > kMaxT) return fail(h, KNNG_ERR_INVALID_ARG, "T = %d", T);
    int r = check_k(h, k, -1);
    if (r) return r;
    if (!ids_in || !dists_in || !ids || !dists) return fail(h, KNNG_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard dg(h->device);
    cudaError_t e = run_merge(n, T, k, ids_in, dists_in, ids, dists, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "merge");
    return KNNG_OK;
}

int knng_propagate(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                   int32_t k, int32_t rounds, const int32_t* ids_in, const float* dists_in,
                   int32_t* ids, float* dists, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_k(h, k, -1))) return r;
    if (rounds < 1 || rounds > 16) return fail(h, KNNG_ERR_INVALID_ARG, "rounds = %d out of [1, 16]", rounds);
    if (!ids_in || !dists_in || !ids || !dists) return fail(h, KNNG_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nk = (size_t)n * k;
    int32_t* bi[2] = {nullptr, nullptr};
    float* bd[2] = {nullptr, nullptr};
    unsigned long long* fl[2] = {nullptr, nullptr};
    if (rounds > 1) {
        Arena m;
        for (int b = 0; b < 2; ++b) { m.take<int32_t>(nk); m.take<float>(nk); m.take<unsigned long long>(n); }
        if ((r = ensure_ws(h, m.off, st))) return r;
        Arena a;
        a.base = h->ws;
        for (int b = 0; b < 2; ++b) {
            bi[b] = a.take<int32_t>(nk);
            bd[b] = a.take<float>(nk);
            fl[b] = a.take<unsigned long long>(n);
        }
    }
    const int32_t* si = ids_in;
    const float* sd = dists_in;
    const unsigned long long* sf = nullptr;  // the input lists count as all new
    for (int rd = 0; rd < rounds; ++rd) {
        const bool last = rd == rounds - 1;
        int32_t* oi = last ? ids : bi[rd & 1];
        float* od = last ? dists : bd[rd & 1];
        unsigned long long* of = last ? nullptr : fl[rd & 1];
        cudaError_t e = run_propagate(x, k, nullptr, si, sd, sf, oi, od, of, st, nullptr, nullptr,
                                      rd < h->prop_stats_rounds ? h->prop_stats + 2 * rd : nullptr);
        if (e != cudaSuccess) return cuda_fail(h, e, "propagate");
        si = oi;
        sd = od;
        sf = of;
    }
    return KNNG_OK;
}

int knng_propagate_best_first(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                              int32_t k, int32_t budget, int32_t rounds, const int32_t* ids_in, int32_t* ids,
                              float* dists, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_k(h, k, -1))) return r;
    if (budget < k || budget > 512) return fail(h, KNNG_ERR_INVALID_ARG, "budget %d out of [k, 512]", budget);
    if (rounds < 1 || rounds > 16) return fail(h, KNNG_ERR_INVALID_ARG, "rounds = %d out of [1, 16]", rounds);
    if (!ids_in || !ids || !dists) return fail(h, KNNG_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nk = (size_t)n * k;
    int32_t* bi[2] = {nullptr, nullptr};
    float* bd[2] = {nullptr, nullptr};
    if (rounds > 1) {
        Arena m;
        for (int b = 0; b < 2; ++b) { m.take<int32_t>(nk); m.take<float>(nk); }
        if ((r = ensure_ws(h, m.off, st))) return r;
        Arena a;
        a.base = h->ws;
        for (int b = 0; b < 2; ++b) { bi[b] = a.take<int32_t>(nk); bd[b] = a.take<float>(nk); }
    }
    const int32_t* si = ids_in;
    for (int rd = 0; rd < rounds; ++rd) {
        const bool last = rd == rounds - 1;
        int32_t* oi = last ? ids : bi[rd & 1];
        float* od = last ? dists : bd[rd & 1];
        const cudaError_t e = run_propagate_best_first(x, k, budget, nullptr, si, oi, od, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "best-first propagation");
        si = oi;
    }
    return KNNG_OK;
}

int knng_propagate_pairwise(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                            int32_t k, int32_t rounds, const int32_t* ids_in, const float* dists_in, int32_t* ids,
                            float* dists, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_k(h, k, -1))) return r;
    if (rounds < 1 || rounds > 16) return fail(h, KNNG_ERR_INVALID_ARG, "rounds = %d out of [1, 16]", rounds);
    if (!ids_in || !dists_in || !ids || !dists) return fail(h, KNNG_ERR_INVALID_ARG, "NULL pointer");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t nk = (size_t)n * k;
    auto carve = [&](Arena& a, int32_t** bi, float** bd, unsigned long long** fl, PairScratch& pw) {
        for (int b = 0; b < 2; ++b) {
            bi[b] = a.take<int32_t>(nk);
            bd[b] = a.take<float>(nk);
            fl[b] = a.take<unsigned long long>(n);
        }
        pairwise_take(a, n, k, pw);
    };
    int32_t* bi[2];
    float* bd[2];
    unsigned long long* fl[2];
    PairScratch pw;
    Arena m;
    carve(m, bi, bd, fl, pw);
    if ((r = ensure_ws(h, m.off, st))) return r;
    Arena a;
    a.base = h->ws;
    carve(a, bi, bd, fl, pw);
    const int32_t* si = ids_in;
    const float* sd = dists_in;
    const unsigned long long* sf = nullptr;  // the input lists count as all new
    for (int rd = 0; rd < rounds; ++rd) {
        const bool last = rd == rounds - 1;
        int32_t* oi = last ? ids : bi[rd & 1];
        float* od = last ? dists : bd[rd & 1];
        unsigned long long* of = last ? nullptr : fl[rd & 1];
        const cudaError_t e = run_propagate_pairwise(x, k, nullptr, si, sd, sf, oi, od, of, pw, h->dev_err, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "pairwise propagation");
        si = oi;
        sd = od;
        sf = of;
    }
    return KNNG_OK;
}

int knng_divisions_used(const knng_handle* h, int32_t* m, float* rates, int32_t cap)
{
    if (!h || !m || cap < 0 || (cap > 0 && !rates)) return KNNG_ERR_INVALID_ARG;
    *m = h->div_used;
    for (int32_t i = 0; i < cap && i < (int32_t)h->div_rates.size(); ++i) rates[i] = h->div_rates[i];
    return KNNG_OK;
}

int knng_build(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
               const knng_params* p, int32_t* ids, float* dists, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_params(h, p, n))) return r;
    if (!ids || !dists) return fail(h, KNNG_ERR_INVALID_ARG, "NULL output");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = ensure_plan(h, n, p->leaf_size, st))) return r;
    Arena m;
    if ((r = build_pipeline(h, h->plan, h->dplan, x, *p, ids, dists, m, st, true, nullptr, true))) return r;
    if ((r = ensure_ws(h, m.off, st))) return r;
    Arena a;
    a.base = h->ws;
    return build_pipeline(h, h->plan, h->dplan, x, *p, ids, dists, a, st, true, nullptr, true);
}

int knng_normalize_rows(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, float* Xn,
                        int64_t ldn, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if (!Xn) return fail(h, KNNG_ERR_INVALID_ARG, "NULL output");
    if (ldn < d) return fail(h, KNNG_ERR_INVALID_ARG, "ldn = %lld < d", (long long)ldn);
    DeviceGuard dg(h->device);
    const cudaError_t e = run_normalize_rows(x, Xn, ldn, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "normalize rows");
    return KNNG_OK;
}

int knng_exact_knn(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                   const int32_t* queries, int64_t nq, int32_t k, int32_t* ids, float* dists,
                   void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_k(h, k, -1))) return r;
    if (nq < 0 || nq >= (int64_t)1 << 31) return fail(h, KNNG_ERR_INVALID_ARG, "nq = %lld", (long long)nq);
    if (nq == 0) return KNNG_OK;
    if (!queries || !ids || !dists) return fail(h, KNNG_ERR_INVALID_ARG, "NULL pointer");
    if (d > 2048) return fail(h, KNNG_ERR_UNSUPPORTED, "exact k-NN supports d <= 2048");
    DeviceGuard dg(h->device);
    cudaError_t e = run_exact_knn(x, queries, (int)nq, k, ids, dists, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "exact k-NN");
    return KNNG_OK;
}

int knng_sync(knng_handle* h, void* stream)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    DeviceGuard dg(h->device);
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "stream synchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "error word");
    if (flag) {
        cudaMemset(h->dev_err, 0, sizeof(int));
        if (flag == 2)
            return fail(h, KNNG_ERR_LIMIT, "pairwise updating: more offers than the buffer holds (4 per list entry); "
                                           "the lists are valid but some offers were dropped");
        return fail(h, KNNG_ERR_TIMEOUT, "a bounded device wait gave up; results of the affected calls are invalid");
    }
    return KNNG_OK;
}

int knng_set_propagation_counters(knng_handle* h, uint64_t* counters, int32_t rounds)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    if (rounds < 0 || (rounds > 0 && !counters)) return fail(h, KNNG_ERR_INVALID_ARG, "bad counters");
    h->prop_stats = rounds > 0 ? reinterpret_cast<unsigned long long*>(counters) : nullptr;
    h->prop_stats_rounds = rounds;
    return KNNG_OK;
}

int knng_set_wait_limit(knng_handle* h, int64_t cycles)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    if (cycles < 0) return fail(h, KNNG_ERR_INVALID_ARG, "wait limit %lld", (long long)cycles);
    h->wait_cycles = cycles;
    return KNNG_OK;
}

int knng_launch_counter(uint64_t* count)
{
    if (!count) return KNNG_ERR_INVALID_ARG;
    *count = launch_count();
    return KNNG_OK;
}

int knng_set_stage_events(knng_handle* h, void* const* events, int32_t nevents)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    if (nevents < 0 || (nevents > 0 && !events)) return fail(h, KNNG_ERR_INVALID_ARG, "bad events");
    h->stage_ev.clear();
    DeviceGuard dg(h->device);
    for (int i = 0; i < nevents; ++i) {
        cudaEvent_t ev = static_cast<cudaEvent_t>(events[i]);
        const cudaError_t e = ev ? cudaEventQuery(ev) : cudaErrorInvalidResourceHandle;
        if (e != cudaSuccess && e != cudaErrorNotReady) {
            cudaGetLastError();
            h->stage_ev.clear();
            return fail(h, KNNG_ERR_INVALID_ARG, "event %d is not a valid CUDA event", i);
        }
        h->stage_ev.push_back(ev);
    }
    return KNNG_OK;
}

int knng_build_batched(knng_handle* h, int32_t nsets, const knng_dataset* sets, const knng_params* p, void* stream)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    if (nsets < 1 || nsets > 65536 || !sets) return fail(h, KNNG_ERR_INVALID_ARG, "nsets = %d", nsets);
    if (!p) return fail(h, KNNG_ERR_INVALID_ARG, "params is NULL");
    if (p->r_stop > 0.f)
        return fail(h, KNNG_ERR_UNSUPPORTED, "adaptive divisions check r_m on the host; a recorded batch cannot");
    int r;
    for (int i = 0; i < nsets; ++i) {
        XDesc x;
        const knng_dataset& D = sets[i];
        if ((r = check_x(h, D.X, D.dtype, D.n, D.d, D.ld, x))) return r;
        if ((r = check_params(h, p, D.n))) return r;
        if (!D.ids || !D.dists) return fail(h, KNNG_ERR_INVALID_ARG, "set %d: NULL output", i);
    }
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BatchCache& B = h->batch;
    std::vector<uint64_t> sig;
    sig.push_back((uint64_t)nsets);
    const uint64_t* pw = reinterpret_cast<const uint64_t*>(p);
    for (size_t i = 0; i < sizeof(knng_params) / 8; ++i) sig.push_back(pw[i]);
    for (int i = 0; i < nsets; ++i) {
        const knng_dataset& D = sets[i];
        sig.push_back((uint64_t)(uintptr_t)D.X);
        sig.push_back(((uint64_t)(uint32_t)D.dtype << 32) | (uint32_t)D.d);
        sig.push_back((uint64_t)D.n);
        sig.push_back((uint64_t)D.ld);
        sig.push_back((uint64_t)(uintptr_t)D.ids);
        sig.push_back((uint64_t)(uintptr_t)D.dists);
    }
    if (!B.cap) {
        if (cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B.ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&B.ev_out, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, KNNG_ERR_CUDA, "batch stream / events");
        }
    }
    if (!B.exec || sig != B.sig) {
        // ---- record the batch: groups of equal (dtype, d) form one forest
        if (B.exec) { cudaGraphExecDestroy(B.exec); B.exec = nullptr; }
        if (B.graph) { cudaGraphDestroy(B.graph); B.graph = nullptr; }
        B.sig.clear();
        B.groups.clear();
        for (int i = 0; i < nsets; ++i) {
            BatchGroup* g = nullptr;
            for (BatchGroup& q : B.groups)
                if (q.dtype == sets[i].dtype && q.d == sets[i].d) g = &q;
            if (!g) {
                B.groups.emplace_back();
                g = &B.groups.back();
                g->dtype = sets[i].dtype;
                g->d = sets[i].d;
                g->ld = (sets[i].d + 3) & ~3;
            }
            g->members.push_back(i);
        }
        // plans and tables (one device buffer for all groups)
        std::vector<char> host;
        auto put = [&](const void* src, size_t bytes) {
            size_t o = (host.size() + 255) & ~(size_t)255;
            host.resize(o + bytes);
            if (bytes) memcpy(host.data() + o, src, bytes);
            return o;
        };
        std::vector<size_t> offs;
        for (BatchGroup& g : B.groups) {
            std::vector<int64_t> roots;
            std::vector<BatchSet> bs;
            int64_t off = 0;
            for (int i : g.members) {
                roots.push_back(sets[i].n);
                bs.push_back(BatchSet{off, sets[i].n, sets[i].ids, sets[i].dists});
                off += sets[i].n;
            }
            g.n = off;
            if (g.n >= (int64_t)1 << 31) return fail(h, KNNG_ERR_UNSUPPORTED, "a group of sets exceeds 2^31 points");
            make_forest_plan(roots, p->leaf_size, g.plan);
            offs.push_back(put(g.plan.nodes.data(), sizeof(SplitNode) * g.plan.nodes.size()));
            offs.push_back(put(g.plan.chunks.data(), sizeof(Chunk) * g.plan.chunks.size()));
            offs.push_back(put(g.plan.leaf_off.data(), sizeof(int32_t) * g.plan.leaf_off.size()));
            offs.push_back(put(bs.data(), sizeof(BatchSet) * bs.size()));
        }
        if (host.size() > B.tables_size) {
            cudaStreamSynchronize(st);
            if (B.tables) cudaFree(B.tables);
            B.tables = nullptr;
            B.tables_size = 0;
            void* q = nullptr;
            if (cudaMalloc(&q, host.size()) != cudaSuccess) {
                cudaGetLastError();
                return fail(h, KNNG_ERR_OOM, "batch tables");
            }
            B.tables = static_cast<char*>(q);
            B.tables_size = host.size();
        } else {
            cudaStreamSynchronize(st);
        }
        if (cudaMemcpy(B.tables, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return cuda_fail(h, cudaGetLastError(), "batch table upload");
        for (size_t gi = 0; gi < B.groups.size(); ++gi) {
            BatchGroup& g = B.groups[gi];
            g.dp.nodes = reinterpret_cast<const SplitNode*>(B.tables + offs[4 * gi + 0]);
            g.dp.chunks = reinterpret_cast<const Chunk*>(B.tables + offs[4 * gi + 1]);
            g.dp.leaf_off = reinterpret_cast<const int32_t*>(B.tables + offs[4 * gi + 2]);
            g.dev_sets = reinterpret_cast<const BatchSet*>(B.tables + offs[4 * gi + 3]);
        }
        // workspace: the largest group (groups run one after another)
        size_t need = 0;
        for (BatchGroup& g : B.groups) {
            Arena m;
            const size_t es = dtype_size(g.dtype);
            m.take<char>((size_t)g.n * g.ld * es);
            m.take<int32_t>((size_t)g.n * p->k);
            m.take<float>((size_t)g.n * p->k);
            XDesc x{nullptr, g.dtype, g.n, g.d, g.ld, true};
            if ((r = build_pipeline(h, g.plan, g.dp, x, *p, nullptr, nullptr, m, st, false))) return r;
            need = std::max(need, m.off);
        }
        if ((r = ensure_ws(h, need, st))) return r;
        if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_fail(h, cudaGetLastError(), "batch setup");
        // record every group's pipeline into one graph
        if (cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return cuda_fail(h, cudaGetLastError(), "begin capture");
        int rr = KNNG_OK;
        const unsigned long long c0 = launch_count();
        for (BatchGroup& g : B.groups) {
            Arena a;
            a.base = h->ws;
            const size_t es = dtype_size(g.dtype);
            char* xc = a.take<char>((size_t)g.n * g.ld * es);
            int32_t* gi = a.take<int32_t>((size_t)g.n * p->k);
            float* gd = a.take<float>((size_t)g.n * p->k);
            int64_t off = 0;
            for (int i : g.members) {
                const knng_dataset& D = sets[i];
                cudaMemcpy2DAsync(xc + (size_t)off * g.ld * es, (size_t)g.ld * es, D.X, (size_t)D.ld * es,
                                  (size_t)D.d * es, (size_t)D.n, cudaMemcpyDeviceToDevice, B.cap);
                off += D.n;
            }
            XDesc x{xc, g.dtype, g.n, g.d, g.ld, true};
            if ((rr = build_pipeline(h, g.plan, g.dp, x, *p, gi, gd, a, B.cap, false))) break;
            if (run_scatter_batch(g.n, p->k, g.dev_sets, (int)g.members.size(), gi, gd, B.cap) != cudaSuccess) {
                rr = cuda_fail(h, cudaGetLastError(), "batch scatter");
                break;
            }
        }
        // kernels recorded into the graph run on replay, not now
        B.kernels = (int)(launch_count() - c0);
        note_launches(-B.kernels);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(B.cap, &graph);
        if (rr) {
            if (graph) cudaGraphDestroy(graph);
            return rr;
        }
        if (ec != cudaSuccess || !graph) return cuda_fail(h, ec, "end capture");
        if (cudaGraphInstantiate(&B.exec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_fail(h, cudaGetLastError(), "graph instantiate");
        }
        B.graph = graph;
        B.sig = sig;
    }
    // ---- one graph launch, ordered after and before the caller's stream
    cudaError_t e = cudaEventRecord(B.ev_in, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B.cap, B.ev_in, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(B.exec, B.cap);
    note_launches(B.kernels);
    if (e == cudaSuccess) e = cudaEventRecord(B.ev_out, B.cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, B.ev_out, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    return KNNG_OK;
}

int knng_autotune(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                  const knng_params* p, int32_t* stages, int32_t* rows_per_group, float* best_ms, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_params(h, p, n))) return r;
    if (p->precision != KNNG_PREC_BF16 && p->precision != KNNG_PREC_FP8E4M3)
        return fail(h, KNNG_ERR_UNSUPPORTED, "tiles are tuned for the tensor-core precisions only");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = ensure_plan(h, n, p->leaf_size, st))) return r;
    const int T = p->T, k = p->k;
    const size_t nk = (size_t)n * k;
    const int kp = std::min(p->rescore_mult * k, 128);
    // perm | lists | max(partition, leaf scratch)
    Arena m;
    m.take<int32_t>((size_t)T * n);
    m.take<int32_t>((size_t)T * nk);
    m.take<float>((size_t)T * nk);
    const size_t fixed = m.off;
    run_partition(x, h->plan, h->dplan, T, p->seed, nullptr, m, st);
    const size_t pe = m.off;
    m.off = fixed;
    run_leaf_knn_tc(x, h->plan, h->dplan, T, nullptr, k, kp, p->precision, nullptr, nullptr, nullptr, m, st);
    if ((r = ensure_ws(h, std::max(pe, m.off), st))) return r;
    Arena a;
    a.base = h->ws;
    int32_t* perm = a.take<int32_t>((size_t)T * n);
    int32_t* li = a.take<int32_t>((size_t)T * nk);
    float* ldd = a.take<float>((size_t)T * nk);
    cudaError_t e = run_partition(x, h->plan, h->dplan, T, p->seed, perm, a, st, nullptr, 0, nullptr, h->dev_err);
    if (e != cudaSuccess) return cuda_fail(h, e, "partition");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    TcTile best_t{};
    for (const TcTile& t : tc_candidates(h->plan, d, p->precision)) {
        float ms = 0.f;
        for (int rep = 0; rep < 4; ++rep) {
            a.off = fixed;
            cudaEventRecord(e0, st);
            e = run_leaf_knn_tc(x, h->plan, h->dplan, T, perm, k, kp, p->precision, li, ldd, h->dev_err, a, st, &t);
            cudaEventRecord(e1, st);
            if (e != cudaSuccess) break;
            cudaEventSynchronize(e1);
            float one = 0.f;
            cudaEventElapsedTime(&one, e0, e1);
            if (rep > 0) ms += one;  // the first run warms up
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (ms < best) {
            best = ms;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_t.S == 0) return fail(h, KNNG_ERR_INTERNAL, "no tile configuration ran");
    h->tune[tc_key(h->plan, d, p->precision)] = best_t;
    if (stages) *stages = best_t.S;
    if (rows_per_group) *rows_per_group = best_t.RG;
    if (best_ms) *best_ms = best / 3.f;
    return knng_sync(h, stream);
}

int knng_tune_save(knng_handle* h, const char* path)
{
    if (!h || !path) return KNNG_ERR_INVALID_ARG;
    FILE* f = fopen(path, "w");
    if (!f) return fail(h, KNNG_ERR_INVALID_ARG, "cannot write %s", path);
    fprintf(f, "# knng tensor-core leaf tiles: precision row_bytes n_load stages rows_per_group\n");
    for (const auto& kv : h->tune)
        fprintf(f, "%d %d %d %d %d\n", kv.first.prec, kv.first.row_bytes, kv.first.n_load, kv.second.S, kv.second.RG);
    fclose(f);
    return KNNG_OK;
}

int knng_tune_load(knng_handle* h, const char* path)
{
    if (!h || !path) return KNNG_ERR_INVALID_ARG;
    FILE* f = fopen(path, "r");
    if (!f) return fail(h, KNNG_ERR_INVALID_ARG, "cannot read %s", path);
    char line[256];
    int added = 0;
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '#') continue;
        TcKey key{};
        TcTile t{};
        if (sscanf(line, "%d %d %d %d %d", &key.prec, &key.row_bytes, &key.n_load, &t.S, &t.RG) == 5 && t.S >= 1 &&
            t.S <= 4 && (t.RG == 32 || t.RG == 64 || t.RG == 128)) {
            h->tune[key] = t;
            ++added;
        }
    }
    fclose(f);
    return KNNG_OK;
}

int knng_mlp_forward(knng_handle* h, knng_mlp* m, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                     float* Z, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    MlpModel* M = mlp_model(m);
    if (!M || !Z) return fail(h, KNNG_ERR_INVALID_ARG, "NULL network or output");
    if (M->d != d) return fail(h, KNNG_ERR_INVALID_ARG, "network input %d != d %d", M->d, d);
    if (d > 128) return fail(h, KNNG_ERR_UNSUPPORTED, "tensor-core inference supports d <= 128");
    DeviceGuard dg(h->device);
    const cudaError_t e = run_mlp_forward(*M, x, Z, h->dev_err, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(h, e, "network inference");
    return KNNG_OK;
}

int knng_build_learned(knng_handle* h, knng_mlp* m, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                       const knng_params* p, int32_t* ids, float* dists, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if (!p) return fail(h, KNNG_ERR_INVALID_ARG, "params is NULL");
    knng_params q = *p;
    // KNNG_PART_FEATURES: per-level learned features (random directions past
    // them); KNNG_PART_RANDOM / KNNG_PART_PCA: random or principal-direction
    // trees in the learned embedding
    const int mode = q.partitioner;
    if (mode != KNNG_PART_FEATURES && mode != KNNG_PART_FEATURES_PCA && mode != KNNG_PART_RANDOM &&
        mode != KNNG_PART_PCA)
        return fail(h, KNNG_ERR_INVALID_ARG, "partitioner %d", mode);
    q.partitioner = (mode == KNNG_PART_PCA || mode == KNNG_PART_FEATURES_PCA) ? KNNG_PART_PCA : KNNG_PART_RANDOM;
    if ((r = check_params(h, &q, n))) return r;
    MlpModel* M = mlp_model(m);
    if (!M || !ids || !dists) return fail(h, KNNG_ERR_INVALID_ARG, "NULL network or output");
    if (M->d != d) return fail(h, KNNG_ERR_INVALID_ARG, "network input %d != d %d", M->d, d);
    if (d > 128) return fail(h, KNNG_ERR_UNSUPPORTED, "tensor-core inference supports d <= 128");
    if (q.metric != KNNG_METRIC_L2) return fail(h, KNNG_ERR_UNSUPPORTED, "learned splits use the L2 metric");
    if (q.T > 32) return fail(h, KNNG_ERR_INVALID_ARG, "T");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = ensure_plan(h, n, q.leaf_size, st))) return r;
    LearnedFeat lf;
    lf.C = M->C;
    learned_feature_order(q.seed, q.T, M->C, lf);
    const bool feat = mode == KNNG_PART_FEATURES || mode == KNNG_PART_FEATURES_PCA;
    XDesc xz{nullptr, KNNG_DTYPE_F32, n, M->C, M->C, true};  // the embedding as the partition's points
    Arena m0;
    m0.take<float>((size_t)n * M->C);
    m0.take<uint32_t>(2 * (size_t)M->C);
    m0.take<float>((size_t)M->C);
    if ((r = build_pipeline(h, h->plan, h->dplan, x, q, ids, dists, m0, st, true, feat ? &lf : nullptr, true,
                            feat ? nullptr : &xz)))
        return r;
    if ((r = ensure_ws(h, m0.off, st))) return r;
    Arena a;
    a.base = h->ws;
    float* Z = a.take<float>((size_t)n * M->C);
    uint32_t* mm = a.take<uint32_t>(2 * (size_t)M->C);
    float* frange = a.take<float>((size_t)M->C);
    lf.Z = Z;
    lf.frange = frange;
    const bool rec = (int)h->stage_ev.size() >= 5 + q.prop_rounds;
    if (rec) cudaEventRecord(h->stage_ev[4 + q.prop_rounds], st);  // start of inference
    cudaError_t e = run_mlp_forward(*M, x, Z, h->dev_err, st);
    if (e == cudaSuccess && feat) e = run_feature_range(Z, n, M->C, mm, frange, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "network inference");
    xz.X = Z;
    return build_pipeline(h, h->plan, h->dplan, x, q, ids, dists, a, st, true, feat ? &lf : nullptr, true,
                          feat ? nullptr : &xz);
}

int knng_partition_learned(knng_handle* h, knng_mlp* m, const void* X, int32_t dtype, int64_t n, int32_t d,
                           int64_t ld, int32_t T, int32_t g, uint64_t seed, int32_t* perm, float* Zout, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if ((r = check_tree(h, T, g))) return r;
    if (!perm) return fail(h, KNNG_ERR_INVALID_ARG, "perm is NULL");
    if (T > 32) return fail(h, KNNG_ERR_INVALID_ARG, "T");
    MlpModel* M = mlp_model(m);
    if (!M) return fail(h, KNNG_ERR_INVALID_ARG, "NULL network");
    if (M->d != d) return fail(h, KNNG_ERR_INVALID_ARG, "network input %d != d %d", M->d, d);
    if (d > 128) return fail(h, KNNG_ERR_UNSUPPORTED, "tensor-core inference supports d <= 128");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = ensure_plan(h, n, g, st))) return r;
    LearnedFeat lf;
    lf.C = M->C;
    learned_feature_order(seed, T, M->C, lf);
    Arena m0;
    if (!Zout) m0.take<float>((size_t)n * M->C);
    m0.take<uint32_t>(2 * (size_t)M->C);
    m0.take<float>((size_t)M->C);
    run_partition(x, h->plan, h->dplan, T, seed, nullptr, m0, st, &lf);
    if ((r = ensure_ws(h, m0.off, st))) return r;
    Arena a;
    a.base = h->ws;
    float* Z = Zout ? Zout : a.take<float>((size_t)n * M->C);
    uint32_t* mm = a.take<uint32_t>(2 * (size_t)M->C);
    float* frange = a.take<float>((size_t)M->C);
    lf.Z = Z;
    lf.frange = frange;
    cudaError_t e = run_mlp_forward(*M, x, Z, h->dev_err, st);
    if (e == cudaSuccess) e = run_feature_range(Z, n, M->C, mm, frange, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "network inference");
    e = run_partition(x, h->plan, h->dplan, T, seed, perm, a, st, &lf, 0, nullptr, h->dev_err);
    if (e != cudaSuccess) return cuda_fail(h, e, "partition");
    return KNNG_OK;
}

int knng_build_host(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                    const knng_params* p, int32_t* ids, float* dists, void* stream)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    if (!X || !ids || !dists || !p) return fail(h, KNNG_ERR_INVALID_ARG, "NULL pointer");
    if (n < 2 || n >= (int64_t)1 << 31 || d < 1 || ld < d || p->k < 1 || p->k > kMaxK)
        return fail(h, KNNG_ERR_INVALID_ARG, "bad sizes");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = dtype_size(dtype);
    const size_t xbytes = (size_t)((n - 1) * ld + d) * es;
    const size_t nk = (size_t)n * p->k;
    // device copies of X and of the graph, kept by the handle between calls
    const size_t xpad = (xbytes + 255) & ~(size_t)255;
    const size_t need = xpad + nk * 8;
    cudaError_t e = cudaSuccess;
    if (need > h->staging_size) {
        if (h->staging) cudaFreeAsync(h->staging, st);
        h->staging = nullptr;
        h->staging_size = 0;
        void* q = nullptr;
        e = cudaMallocAsync(&q, need, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, KNNG_ERR_OOM, "staging buffers");
        }
        h->staging = static_cast<char*>(q);
        h->staging_size = need;
    }
    void* dx = h->staging;
    int32_t* di = reinterpret_cast<int32_t*>(h->staging + xpad);
    float* dd = reinterpret_cast<float*>(di + nk);
    int r = KNNG_OK;
    e = cudaMemcpyAsync(dx, X, xbytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) r = cuda_fail(h, e, "copy X to device");
    if (!r) r = knng_build(h, dx, dtype, n, d, ld, p, di, dd, stream);
    if (!r) {
        e = cudaMemcpyAsync(ids, di, nk * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dists, dd, nk * 4, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) r = cuda_fail(h, e, "copy graph to host");
    }
    const int rs = knng_sync(h, stream);
    return r ? r : rs;
}

}  // extern "C"
