// Random principal directions (Sec. 3.4 of arXiv:1307.7852, "Random
// division": a node is split along the principal direction of points
// sampled at random from it, computed by the Lanczos algorithm).
//
// One block per split node of a level (grid: nodes x trees):
//  1. sample: a node of m points with m <= s_cap takes all of them, else
//     s_cap members M[w_r mod m] (w_r: word r mod 4 of Philox4x32-10 with
//     counter (tree, level | 2^30, node, r / 4)); members are read in the
//     node's ascending-id order; s_cap = clamp(floor(40960 / d), 8, 128);
//  2. the sampled rows, centred, in shared memory (FP32);
//  3. Lanczos with full reorthogonalisation (one classical Gram-Schmidt
//     pass of C v_j against every earlier basis vector, whose coefficient
//     on v_j is alpha_j) on C = A^T A / s from the node's random direction,
//     at most min(8, d) steps, stopping once beta_j <= 1e-4 * max alpha;
//  4. the top eigenvector of the tridiagonal matrix (one warp: Sturm
//     multisection for the eigenvalue, inverse iteration for the vector),
//     the Ritz vector, normalised, its largest entry made positive (ties:
//     the lowest index).
// The direction replaces the node's random direction before the projection
// (the split itself is unchanged) and is optionally written out by
// (level, node) for replay.
#include "knng_common.cuh"
#include "knng_internal.h"

#include <type_traits>

namespace knng {

namespace {
constexpr int kPcaThreads = 256;
constexpr int kPcaSteps = 8;
constexpr uint32_t kPcaLevelTag = 1u << 30;
}  // namespace

__host__ __device__ inline int pca_sample_cap(int d)
{
    int s = 40960 / d;
    s = s > 128 ? 128 : s;
    return s < 8 ? 8 : s;
}

size_t pca_smem_bytes(int d)
{
    const int dp = (d + 3) & ~3;
    const int s = pca_sample_cap(d);
    return sizeof(float) * ((size_t)s * dp + (size_t)(kPcaSteps + 1) * dp + 2 * (size_t)dp + 128 +
                            (kPcaThreads / 32) * kPcaSteps + 8);
}

// Number of eigenvalues of the symmetric tridiagonal matrix (alpha, beta)
// below x (Sturm sequence of the LDL^T pivots).
__device__ __forceinline__ int sturm_below(const float* alpha, const float* beta, int q, float x)
{
    int c = 0;
    float dv = 1.f;
    for (int i = 0; i < q; ++i) {
        const float b2 = i > 0 ? beta[i - 1] * beta[i - 1] : 0.f;
        dv = (alpha[i] - x) - (i > 0 ? b2 / dv : 0.f);
        if (dv == 0.f) dv = -1e-30f;
        c += dv < 0.f ? 1 : 0;
    }
    return c;
}

// Top eigenvector of the symmetric tridiagonal q x q matrix (alpha, beta),
// q <= 8, by one warp: the largest eigenvalue by 33-way multisection of the
// Gershgorin interval on Sturm counts, then two steps of inverse iteration
// (tridiagonal elimination) on lane 0.  y: q entries (not normalised).
__device__ void tridiag_top(const float* alpha, const float* beta, int q, float* y)
{
    const int lane = threadIdx.x & 31;
    float lo = 3.4e38f, hi = -3.4e38f;
    for (int i = 0; i < q; ++i) {
        const float r = (i > 0 ? fabsf(beta[i - 1]) : 0.f) + (i + 1 < q ? fabsf(beta[i]) : 0.f);
        lo = fminf(lo, alpha[i] - r);
        hi = fmaxf(hi, alpha[i] + r);
    }
    hi += 1e-6f * (fabsf(hi) + fabsf(lo)) + 1e-30f;
    for (int it = 0; it < 8; ++it) {
        const float x = lo + (hi - lo) * (float)(lane + 1) / 33.f;
        const bool above = sturm_below(alpha, beta, q, x) == q;  // x above every eigenvalue
        const uint32_t m = __ballot_sync(KNNG_FULL_MASK, above);
        const int first = m ? __ffs(m) - 1 : 32;
        const float nhi = first < 32 ? lo + (hi - lo) * (float)(first + 1) / 33.f : hi;
        const float nlo = lo + (hi - lo) * (float)first / 33.f;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0) {
        const float lam = 0.5f * (lo + hi);
        float v[8], dd[8], cc[8];
        for (int i = 0; i < q; ++i) v[i] = 1.f;
        for (int rep = 0; rep < 2; ++rep) {
            // solve (T - lam I) z = v by elimination without pivoting
            for (int i = 0; i < q; ++i) {
                float piv = alpha[i] - lam - (i > 0 ? beta[i - 1] * cc[i - 1] : 0.f);
                if (fabsf(piv) < 1e-30f) piv = 1e-30f;
                cc[i] = i + 1 < q ? beta[i] / piv : 0.f;
                dd[i] = (v[i] - (i > 0 ? beta[i - 1] * dd[i - 1] : 0.f)) / piv;
            }
            for (int i = q - 1; i >= 0; --i) v[i] = dd[i] - (i + 1 < q ? cc[i] * v[i + 1] : 0.f);
            float nn = 0.f;
            for (int i = 0; i < q; ++i) nn = fmaxf(nn, fabsf(v[i]));
            for (int i = 0; i < q; ++i) v[i] /= nn;
        }
        for (int i = 0; i < q; ++i) y[i] = v[i];
    }
    __syncwarp();
}

// Sums of cnt per-thread values over the block (fixed order); red holds
// (threads / 32) * kPcaSteps + 8 floats.
template <int N>
__device__ __forceinline__ void pca_block_sums(float (&v)[N], int cnt, float* red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i < cnt) {
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) v[i] += __shfl_xor_sync(KNNG_FULL_MASK, v[i], o);
        }
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < cnt) red[w * N + i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
        if (i < cnt) {
            float s = 0.f;
            for (int ww = 0; ww < kPcaThreads / 32; ++ww) s += red[ww * N + i];
            v[i] = s;
        }
    }
}

template <class Loader>
__device__ void pca_node(const Loader& L, int64_t n, const SplitNode& nd, const int32_t* __restrict__ cur, int t,
                         uint32_t level, uint64_t seed, uint32_t t0, int dp, float* __restrict__ dir,
                         float* __restrict__ out)
{
    extern __shared__ __align__(16) float sm[];
    const int d = L.d;
    const int cap = pca_sample_cap(d);
    const int m = nd.size;
    const int s = m <= cap ? m : cap;
    float* A = sm;                          // s x dp, centred sample
    float* V = A + (size_t)cap * dp;        // (kPcaSteps + 1) x dp, Lanczos basis
    float* w = V + (size_t)(kPcaSteps + 1) * dp;
    float* mu = w + dp;
    float* u = mu + dp;                     // s <= 128
    float* red = u + 128;                   // 8 warp partials (+ spare)
    __shared__ int rows[128];
    __shared__ float alpha[kPcaSteps], beta[kPcaSteps];
    __shared__ float ysh[kPcaSteps];
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;

    // 1. sample
    const int32_t* mem = cur + (int64_t)t * n + nd.off;
    const uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    for (int r = tid; r < s; r += kPcaThreads) {
        int idx = r;
        if (m > cap) {
            const uint4 q4 = philox4x32_10(make_uint4(t0 + (uint32_t)t, level | kPcaLevelTag, nd.v, (uint32_t)(r >> 2)),
                                           key);
            const uint32_t word = (r & 3) == 0 ? q4.x : (r & 3) == 1 ? q4.y : (r & 3) == 2 ? q4.z : q4.w;
            idx = (int)(word % (uint32_t)m);
        }
        rows[r] = mem[idx];
    }
    __syncthreads();
    // 2. rows, mean, centring
    if (L.all_vec()) {
        const int d4 = d >> 2;
        for (int e = tid; e < s * d4; e += kPcaThreads) {
            const int r = e / d4, j = 4 * (e - (e / d4) * d4);
            *reinterpret_cast<float4*>(A + (size_t)r * dp + j) = L.load4v(rows[r], j);
        }
    } else {
        for (int e = tid; e < s * d; e += kPcaThreads) {
            const int r = e / d, j = e - (e / d) * d;
            A[(size_t)r * dp + j] = L.load1(rows[r], j);
        }
    }
    __syncthreads();
    for (int j = tid; j < d; j += kPcaThreads) {
        float acc = 0.f;
        for (int r = 0; r < s; ++r) acc += A[(size_t)r * dp + j];
        mu[j] = acc / (float)s;
    }
    __syncthreads();
    for (int e = tid; e < s * d; e += kPcaThreads) {
        const int r = e / d, j = e - (e / d) * d;
        A[(size_t)r * dp + j] -= mu[j];
    }
    // start vector: the node's random direction, normalised
    float v1[1] = {0.f};
    for (int j = tid; j < d; j += kPcaThreads) {
        const float x = dir[j];
        V[j] = x;
        v1[0] = fmaf(x, x, v1[0]);
    }
    pca_block_sums(v1, 1, red);
    const float nv = sqrtf(v1[0]);
    for (int j = tid; j < d; j += kPcaThreads) V[j] /= nv;
    __syncthreads();

    // 3. Lanczos with full reorthogonalisation
    const int steps = d < kPcaSteps ? d : kPcaSteps;
    float amax = 0.f;
    int q = 0;
    for (int j = 0; j < steps; ++j) {
        const float* vj = V + (size_t)j * dp;
        // u = A v_j (one warp per row, lane partials + butterfly)
        for (int r = wp; r < s; r += kPcaThreads / 32) {
            float acc = 0.f;
            for (int c = lane; c < d; c += 32) acc = fmaf(A[(size_t)r * dp + c], vj[c], acc);
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(KNNG_FULL_MASK, acc, o);
            if (lane == 0) u[r] = acc;
        }
        __syncthreads();
        // w = A^T u / s; one classical Gram-Schmidt pass against v_0 .. v_j
        // (full reorthogonalisation) gives alpha_j, the coefficient of v_j,
        // and removes the three-term recurrence's part with the rest
        float coef[kPcaSteps];
#pragma unroll
        for (int i = 0; i < kPcaSteps; ++i) coef[i] = 0.f;
        for (int c = tid; c < d; c += kPcaThreads) {
            float acc = 0.f;
            for (int r = 0; r < s; ++r) acc = fmaf(A[(size_t)r * dp + c], u[r], acc);
            const float wc = acc / (float)s;
            w[c] = wc;
#pragma unroll
            for (int i = 0; i < kPcaSteps; ++i)
                if (i <= j) coef[i] = fmaf(V[(size_t)i * dp + c], wc, coef[i]);
        }
        pca_block_sums(coef, j + 1, red);
        float a = 0.f;
#pragma unroll
        for (int i = 0; i < kPcaSteps; ++i)
            if (i == j) a = coef[i];
        amax = fmaxf(amax, a);
        v1[0] = 0.f;
        for (int c = tid; c < d; c += kPcaThreads) {
            float x = w[c];
#pragma unroll
            for (int i = 0; i < kPcaSteps; ++i)
                if (i <= j) x -= coef[i] * V[(size_t)i * dp + c];
            w[c] = x;
            v1[0] = fmaf(x, x, v1[0]);
        }
        pca_block_sums(v1, 1, red);
        const float b = sqrtf(v1[0]);
        if (tid == 0) {
            alpha[j] = a;
            beta[j] = b;
        }
        q = j + 1;
        if (j == steps - 1 || b <= 1e-4f * amax) break;
        for (int c = tid; c < d; c += kPcaThreads) V[(size_t)(j + 1) * dp + c] = w[c] / b;
        __syncthreads();
    }
    __syncthreads();
    // 4. tridiagonal eigenvector (one warp), Ritz vector
    if (wp == 0) tridiag_top(alpha, beta, q, ysh);
    __syncthreads();
    v1[0] = 0.f;
    for (int c = tid; c < d; c += kPcaThreads) {
        float x = 0.f;
        for (int i = 0; i < q; ++i) x = fmaf(ysh[i], V[(size_t)i * dp + c], x);
        w[c] = x;
        v1[0] = fmaf(x, x, v1[0]);
    }
    pca_block_sums(v1, 1, red);
    const float nrm = sqrtf(v1[0]);
    // sign: the largest-magnitude entry positive (ties: the lowest index)
    float best = -1.f;
    int bi = 0x7FFFFFFF;
    for (int c = tid; c < d; c += kPcaThreads) {
        const float av = fabsf(w[c]);
        if (av > best) {
            best = av;
            bi = c;
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const float ob = __shfl_xor_sync(KNNG_FULL_MASK, best, o);
        const int oi = __shfl_xor_sync(KNNG_FULL_MASK, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    __shared__ float bbest[kPcaThreads / 32];
    __shared__ int bidx[kPcaThreads / 32];
    if (lane == 0) {
        bbest[wp] = best;
        bidx[wp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
        for (int i = 1; i < kPcaThreads / 32; ++i)
            if (bbest[i] > bbest[0] || (bbest[i] == bbest[0] && bidx[i] < bidx[0])) {
                bbest[0] = bbest[i];
                bidx[0] = bidx[i];
            }
    }
    __syncthreads();
    const float sgn = w[bidx[0]] < 0.f ? -1.f : 1.f;
    for (int c = tid; c < dp; c += kPcaThreads) {
        const float x = c < d ? sgn * w[c] / nrm : 0.f;
        dir[c] = x;
        if (out && c < d) out[c] = x;
    }
}

template <int kDT>
__global__ void __launch_bounds__(kPcaThreads) pca_dirs_kernel(RowLoader<kDT> L, RowLoader<kDtU8> Lb,
                                                               const int* __restrict__ xb_bad, int64_t n,
                                                               const SplitNode* __restrict__ nodes,
                                                               const int32_t* __restrict__ cur, int S, int dp,
                                                               uint32_t level, uint64_t seed, uint32_t t0,
                                                               float* __restrict__ dirs, float* __restrict__ out,
                                                               int64_t out_tree_stride)
{
    const int sn = blockIdx.x, t = blockIdx.y;
    const SplitNode nd = nodes[sn];
    float* dir = dirs + ((int64_t)t * S + sn) * dp;
    float* o = out ? out + (int64_t)t * out_tree_stride + ((((int64_t)1 << level) - 1) + nd.v) * L.d : nullptr;
    bool bytes = false;
    if constexpr (kDT == kDtF32) bytes = xb_bad && *xb_bad == 0;
    if (kDT == kDtF32 && bytes) pca_node(Lb, n, nd, cur, t, level, seed, t0, dp, dir, o);
    else pca_node(L, n, nd, cur, t, level, seed, t0, dp, dir, o);
}

cudaError_t run_pca_dirs(const XDesc& x, int T, int S, const SplitNode* nodes, const int32_t* cur, int dp,
                         uint32_t level, uint64_t seed, int t0, float* dirs, float* out, int64_t out_tree_stride,
                         cudaStream_t st)
{
    if (x.d > 1024) return cudaErrorInvalidValue;
    const size_t smem = pca_smem_bytes(x.d);
    cudaError_t e = cudaSuccess;
    auto launch = [&](auto dt) {
        constexpr int kDT = decltype(dt)::value;
        auto kern = pca_dirs_kernel<kDT>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return;
        RowLoader<kDT> rl{x.X, x.ld, x.d, x.vec};
        const RowLoader<kDtU8> rb{x.Xb, x.ldb, x.d, true};
        kern<<<dim3(S, T), kPcaThreads, smem, st>>>(rl, rb, x.xb_bad, x.n, nodes, cur, S, dp, level, seed,
                                                    (uint32_t)t0, dirs, out, out_tree_stride);
        note_launches(1);
        e = cudaGetLastError();
    };
    if (x.dtype == kDtF16) launch(std::integral_constant<int, kDtF16>{});
    else if (x.dtype == kDtU8) launch(std::integral_constant<int, kDtU8>{});
    else launch(std::integral_constant<int, kDtF32>{});
    return e;
}

}  // namespace knng
