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
    std::string err;
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

int check_x(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, XDesc& x)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    if (!X) return fail(h, KNNG_ERR_INVALID_ARG, "X is NULL");
    if (dtype != KNNG_DTYPE_F32 && dtype != KNNG_DTYPE_F16) return fail(h, KNNG_ERR_INVALID_ARG, "dtype %d", dtype);
    if (n < 2 || n >= (int64_t)1 << 31) return fail(h, KNNG_ERR_INVALID_ARG, "n = %lld out of [2, 2^31)", (long long)n);
    if (d < 1 || d > 4096) return fail(h, KNNG_ERR_INVALID_ARG, "d = %d out of [1, 4096]", d);
    if (ld < d || ld >= (int64_t)1 << 31) return fail(h, KNNG_ERR_INVALID_ARG, "ld = %lld out of [d, 2^31)", (long long)ld);
    const size_t es = dtype == KNNG_DTYPE_F16 ? 2 : 4;
    const size_t align = dtype == KNNG_DTYPE_F16 ? 8 : 16;
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
int leaf_stage(knng_handle* h, const XDesc& x, int T, const int32_t* perm, int k, int prec, int mult,
               int32_t* ids, float* dists, Arena& ar, cudaStream_t st)
{
    cudaError_t e;
    const int kp = std::min(mult * k, 128);
    if (prec == KNNG_PREC_FP32) {
        if (!ar.base) return KNNG_OK;
        e = run_leaf_knn_f32(x, h->plan, h->dplan, T, perm, k, kp, ids, dists, st);
    } else if (prec == KNNG_PREC_BF16 || prec == KNNG_PREC_FP8E4M3) {
        e = run_leaf_knn_tc(x, h->plan, h->dplan, T, perm, k, kp, prec, ids, dists, h->dev_err, ar, st);
    } else {
        return fail(h, KNNG_ERR_INVALID_ARG, "precision %d", prec);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "leaf k-NN");
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
    cudaError_t e = run_partition(x, h->plan, h->dplan, T, seed, perm, a, st);
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
    if ((r = leaf_stage(h, x, T, perm, k, precision, rescore_mult, ids, dists, m, st))) return r;
    if ((r = ensure_ws(h, m.off, st))) return r;
    Arena a;
    a.base = h->ws;
    return leaf_stage(h, x, T, perm, k, precision, rescore_mult, ids, dists, a, st);
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
        cudaError_t e = run_propagate(x, k, nullptr, si, sd, sf, oi, od, of, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "propagate");
        si = oi;
        sd = od;
        sf = of;
    }
    return KNNG_OK;
}

int knng_build(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
               const knng_params* p, int32_t* ids, float* dists, void* stream)
{
    XDesc x;
    int r = check_x(h, X, dtype, n, d, ld, x);
    if (r) return r;
    if (!p) return fail(h, KNNG_ERR_INVALID_ARG, "params is NULL");
    if ((r = check_tree(h, p->T, p->leaf_size))) return r;
    if ((r = check_k(h, p->k, n > p->leaf_size ? p->leaf_size : -1))) return r;
    if (p->prop_rounds < 0 || p->prop_rounds > 16) return fail(h, KNNG_ERR_INVALID_ARG, "prop_rounds %d", p->prop_rounds);
    if (p->rescore_mult < 1 || p->rescore_mult > 4) return fail(h, KNNG_ERR_INVALID_ARG, "rescore_mult %d", p->rescore_mult);
    if (p->partitioner != KNNG_PART_RANDOM) return fail(h, KNNG_ERR_UNSUPPORTED, "partitioner %d", p->partitioner);
    if (p->reserved != 0) return fail(h, KNNG_ERR_INVALID_ARG, "reserved must be 0");
    if (!ids || !dists) return fail(h, KNNG_ERR_INVALID_ARG, "NULL output");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((r = ensure_plan(h, n, p->leaf_size, st))) return r;
    const int T = p->T, k = p->k;
    const size_t nk = (size_t)n * k;
    // workspace: perm | leaf lists | propagation buffers | max(partition, leaf scratch)
    Arena m;
    m.take<int32_t>((size_t)T * n);
    m.take<int32_t>((size_t)T * nk);
    m.take<float>((size_t)T * nk);
    for (int b = 0; b < 2; ++b) { m.take<int32_t>(nk); m.take<float>(nk); m.take<unsigned long long>(n); }
    const size_t fixed = m.off;
    run_partition(x, h->plan, h->dplan, T, p->seed, nullptr, m, st);
    const size_t part_end = m.off;
    m.off = fixed;
    if ((r = leaf_stage(h, x, T, nullptr, k, p->precision, p->rescore_mult, nullptr, nullptr, m, st))) return r;
    const size_t total = std::max(part_end, m.off);
    if ((r = ensure_ws(h, total, st))) return r;
    Arena a;
    a.base = h->ws;
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
    const size_t fixed2 = a.off;
    const int R = p->prop_rounds;
    const bool rec = (int)h->stage_ev.size() >= 4 + R;
    auto mark = [&](int i) {
        if (rec) cudaEventRecord(h->stage_ev[i], st);
    };
    mark(0);
    cudaError_t e = run_partition(x, h->plan, h->dplan, T, p->seed, perm, a, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "partition");
    mark(1);
    a.off = fixed2;  // the partition scratch is dead: the leaf stage reuses it
    if ((r = leaf_stage(h, x, T, perm, k, p->precision, p->rescore_mult, li, ld_, a, st))) return r;
    mark(2);
    int32_t* mi = R == 0 ? ids : bi[0];
    float* md = R == 0 ? dists : bd[0];
    e = run_merge(n, T, k, li, ld_, mi, md, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "merge");
    mark(3);
    // propagation visits points in the leaf order of tree 0: neighbouring
    // points run together, so candidate rows are shared through L2.
    for (int rd = 0; rd < R; ++rd) {
        const int32_t* si = bi[rd & 1];
        const float* sd = bd[rd & 1];
        const unsigned long long* sf = rd == 0 ? nullptr : fl[rd & 1];
        int32_t* oi = rd == R - 1 ? ids : bi[(rd + 1) & 1];
        float* od = rd == R - 1 ? dists : bd[(rd + 1) & 1];
        unsigned long long* of = rd == R - 1 ? nullptr : fl[(rd + 1) & 1];
        e = run_propagate(x, k, perm, si, sd, sf, oi, od, of, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "propagate");
        mark(4 + rd);
    }
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
        return fail(h, KNNG_ERR_TIMEOUT, "a bounded device wait gave up; results of the affected calls are invalid");
    }
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

int knng_build_host(knng_handle* h, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld,
                    const knng_params* p, int32_t* ids, float* dists, void* stream)
{
    if (!h) return KNNG_ERR_INVALID_ARG;
    if (!X || !ids || !dists || !p) return fail(h, KNNG_ERR_INVALID_ARG, "NULL pointer");
    if (n < 2 || n >= (int64_t)1 << 31 || d < 1 || ld < d || p->k < 1 || p->k > kMaxK)
        return fail(h, KNNG_ERR_INVALID_ARG, "bad sizes");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = dtype == KNNG_DTYPE_F16 ? 2 : 4;
    const size_t xbytes = (size_t)((n - 1) * ld + d) * es;
    const size_t nk = (size_t)n * p->k;
    void* dx = nullptr;
    void* dout = nullptr;
    cudaError_t e = cudaMallocAsync(&dx, xbytes, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&dout, nk * 8, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (dx) cudaFreeAsync(dx, st);
        return fail(h, KNNG_ERR_OOM, "staging buffers");
    }
    int32_t* di = static_cast<int32_t*>(dout);
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
    cudaFreeAsync(dx, st);
    cudaFreeAsync(dout, st);
    const int rs = knng_sync(h, stream);
    return r ? r : rs;
}

}  // extern "C"
