// Learned partitioner: training of the split-feature network.
//
// The paper splits along random principal directions (Sec. 3.4) or random
// projections (appendix after Lemma 1); this library can also split along
// learned features: a network x -> z in (-1, 1)^C (d -> H -> C, GELU, output
// tanh), where level
// l of tree t splits every node at the median of feature pi_t(l).  The
// network is trained on edges (i, j) of k-NN graphs built by the method
// itself, to keep neighbours on the same side of those medians:
//
//   L = sum_c mean_b (z_c(i_b) - z_c(j_b))^2 / (V_c + eps)
//       + lam * sum_{c != c'} corr(z_c, z_c')^2 + mu * sum_c (1 - V_c)^2
// (batch statistics; the last term stops an output from collapsing to a
// constant, which would zero the first two)
//
// All training arithmetic is FP32 in the kernels below: batch sampling
// (Philox), forward and backward GEMMs (tiled SIMT), the loss and its
// gradient through the batch statistics, and Adam.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "../../include/knng.h"
#include "knng_common.cuh"
#include "knng_internal.h"

namespace knng {

// ---------------------------------------------------------------------------
// Tiled FP32 GEMM: C[M][N] (+)= sum_k A(m, k) B(k, n) with A(m, k) = TA ?
// A[k*lda + m] : A[m*lda + k] and B(k, n) = TB ? B[n*ldb + k] : B[k*ldb + n].
// Epilogue: EPI 0 plain store, 1 = + bias[n], store pre-activation to aux and
// GELU to C, 2 = + bias[n], 3 = tanh(. + bias[n]).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float gelu_f(float a)
{
    return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float a)
{
    return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * __expf(-0.5f * a * a);
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                   const float* __restrict__ B, int ldb, float* __restrict__ C,
                                                   int ldc, const float* __restrict__ bias, float* __restrict__ aux)
{
    constexpr int TM = 64, TN = 64, TK = 16;
    __shared__ float As[TK][TM + 4];
    __shared__ float Bs[TK][TN + 4];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += TK) {
        for (int e = tid; e < TM * TK; e += 256) {
            const int mm = TA ? e % TM : e / TK, kk = TA ? e / TM : e % TK;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? (TA ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k]) : 0.f;
        }
        for (int e = tid; e < TN * TK; e += 256) {
            const int nn = TB ? e / TK : e % TN, kk = TB ? e % TK : e / TN;
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < N && k < K) ? (TB ? B[(int64_t)n * ldb + k] : B[(int64_t)k * ldb + n]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m >= M || n >= N) continue;
            float v = acc[i][j];
            if (EPI == 1) {
                v += bias[n];
                aux[(int64_t)m * ldc + n] = v;
                v = gelu_f(v);
            } else if (EPI == 2) {
                v += bias[n];
            } else if (EPI == 3) {
                v = tanhf(v + bias[n]);
            }
            C[(int64_t)m * ldc + n] = v;
        }
}

template <bool TA, bool TB, int EPI>
static void gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                 const float* bias, float* aux, cudaStream_t st)
{
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    gemm_kernel<TA, TB, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, aux);
    note_launches(1);
}

// ---------------------------------------------------------------------------
// Batch sampling: edge b takes a Philox-random point i and a random valid
// slot of its list; row b of Xb is x_i, row B + b is x_j (FP32).
// ---------------------------------------------------------------------------
template <int kDT>
__global__ void sample_batch_kernel(RowLoader<kDT> L, int64_t n, const int32_t* __restrict__ ids, int k, int B,
                                    uint64_t seed, uint32_t step, float* __restrict__ Xb)
{
    const int lane = threadIdx.x & 31;
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= B) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)b, step, 0x4C4E4E42u, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const int64_t i = (int64_t)(((uint64_t)w.x << 32 | w.y) % (uint64_t)n);
    int32_t j = -1;
    for (int t = 0; t < k && j < 0; ++t) {
        const int slot = (int)((w.z + (uint32_t)t) % (uint32_t)k);
        j = ids[i * k + slot];
    }
    if (j < 0 || j >= n) j = (int32_t)i;
    for (int c = 4 * lane; c < L.d; c += 128) {
        const float4 a = L.load4(i, c), v = L.load4(j, c);
        const float av[4] = {a.x, a.y, a.z, a.w}, vv[4] = {v.x, v.y, v.z, v.w};
        for (int e = 0; e < 4 && c + e < L.d; ++e) {
            Xb[(int64_t)b * L.d + c + e] = av[e];
            Xb[(int64_t)(B + b) * L.d + c + e] = vv[e];
        }
    }
}

// ---------------------------------------------------------------------------
// Loss and dL/dZ through the batch statistics (one block).  Z: N x C rows,
// N = 2B.  Writes the loss to *loss and the gradient to dZ.
// ---------------------------------------------------------------------------
constexpr int kLossThreads = 1024;

__global__ void __launch_bounds__(kLossThreads) loss_kernel(const float* __restrict__ Z, int N, int C, float lam,
                                                            float eps, float mus, float* __restrict__ dZ,
                                                            float* __restrict__ loss)
{
    extern __shared__ float sh[];
    float* mu = sh;               // C
    float* var = mu + C;          // C
    float* P = var + C;           // C
    float* Kc = P + C;            // C*C
    float* m1 = Kc + C * C;       // C
    float* m2 = m1 + C;           // C
    float* red = m2 + C;          // kLossThreads
    const int tid = threadIdx.x;
    const int B = N / 2;
    // per-column reductions: thread t handles column t % C over rows r = t / C, ...
    const int per = kLossThreads / C;  // threads per column (C divides 1024)
    const int c = tid % C, r0 = tid / C;
    auto col_reduce = [&](float v) -> float {
        red[tid] = v;
        __syncthreads();
        float s = 0.f;
        if (tid < C)
            for (int q = 0; q < per; ++q) s += red[q * C + tid];
        __syncthreads();
        return s;  // valid for tid < C
    };
    float s = 0.f;
    for (int r = r0; r < N; r += per) s += Z[(int64_t)r * C + c];
    s = col_reduce(s);
    if (tid < C) mu[tid] = s / N;
    __syncthreads();
    float sv = 0.f, sp = 0.f;
    for (int r = r0; r < N; r += per) {
        const float zc = Z[(int64_t)r * C + c] - mu[c];
        sv += zc * zc;
        if (r < B) {
            const float dd = Z[(int64_t)r * C + c] - Z[(int64_t)(r + B) * C + c];
            sp += dd * dd;
        }
    }
    sv = col_reduce(sv);
    if (tid < C) var[tid] = sv / N;
    sp = col_reduce(sp);
    if (tid < C) P[tid] = sp / B;
    __syncthreads();
    // correlation matrix: pair (a, b) of columns, threads split the rows
    const int pairs = C * C;
    const int tpp = kLossThreads / pairs > 0 ? kLossThreads / pairs : 1;
    for (int pr = tid / tpp; pr < pairs; pr += kLossThreads / tpp) {
        const int a = pr / C, bb = pr % C;
        const float sa = rsqrtf(var[a] + eps), sb = rsqrtf(var[bb] + eps);
        float acc = 0.f;
        for (int r = tid % tpp; r < N; r += tpp)
            acc += (Z[(int64_t)r * C + a] - mu[a]) * sa * (Z[(int64_t)r * C + bb] - mu[bb]) * sb;
        // tpp divides 32: reduce inside the thread group
        for (int o = tpp / 2; o >= 1; o >>= 1) acc += __shfl_down_sync(KNNG_FULL_MASK, acc, o, tpp);
        if (tid % tpp == 0) Kc[pr] = acc / N;
    }
    __syncthreads();
    if (tid == 0) {
        float L = 0.f;
        for (int a = 0; a < C; ++a) L += P[a] / (var[a] + eps);
        float Ld = 0.f;
        for (int a = 0; a < C; ++a)
            for (int bb = 0; bb < C; ++bb)
                if (a != bb) Ld += Kc[a * C + bb] * Kc[a * C + bb];
        float Ls = 0.f;
        for (int a = 0; a < C; ++a) Ls += (1.f - var[a]) * (1.f - var[a]);
        *loss = L + lam * Ld + mus * Ls;
    }
    // dS = (2/N) S G with G = 2 lam offdiag(K); then the column means
    float d1 = 0.f, d2 = 0.f;
    for (int r = r0; r < N; r += per) {
        float ds = 0.f;
        for (int a = 0; a < C; ++a) {
            if (a == c) continue;
            const float sa = (Z[(int64_t)r * C + a] - mu[a]) * rsqrtf(var[a] + eps);
            ds += sa * 2.f * lam * Kc[a * C + c];
        }
        ds *= 2.f / N;
        const float sc = (Z[(int64_t)r * C + c] - mu[c]) * rsqrtf(var[c] + eps);
        d1 += ds;
        d2 += ds * sc;
    }
    d1 = col_reduce(d1);
    if (tid < C) m1[tid] = d1 / N;
    d2 = col_reduce(d2);
    if (tid < C) m2[tid] = d2 / N;
    __syncthreads();
    for (int r = r0; r < N; r += per) {
        const float ve = var[c] + eps;
        const float sig = sqrtf(ve);
        const float zc = Z[(int64_t)r * C + c] - mu[c];
        float g = (-P[c] / (ve * ve) - 2.f * mus * (1.f - var[c])) * (2.f / N) * zc;
        const int rb = r < B ? r : r - B;
        const float dd = Z[(int64_t)rb * C + c] - Z[(int64_t)(rb + B) * C + c];
        g += (r < B ? 1.f : -1.f) * (1.f / ve) * (2.f / B) * dd;
        float ds = 0.f;
        for (int a = 0; a < C; ++a) {
            if (a == c) continue;
            const float sa = (Z[(int64_t)r * C + a] - mu[a]) * rsqrtf(var[a] + eps);
            ds += sa * 2.f * lam * Kc[a * C + c];
        }
        ds *= 2.f / N;
        const float sc = zc / sig;
        g += (ds - m1[c] - sc * m2[c]) / sig;
        dZ[(int64_t)r * C + c] = g;
    }
}

// through the output tanh: dZpre = dZ (1 - Z^2)
__global__ void tanh_back_kernel(int64_t count, const float* __restrict__ Z, float* __restrict__ dZ)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        dZ[e] *= 1.f - Z[e] * Z[e];
}

// dA = dH * GELU'(A)
__global__ void gelu_back_kernel(int64_t count, const float* __restrict__ A, float* __restrict__ dH)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        dH[e] *= gelu_grad_f(A[e]);
}

// column sums: out[n] = sum_m X[m][n]
__global__ void colsum_kernel(int M, int N, const float* __restrict__ X, float* __restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += X[(int64_t)m * N + n];
    out[n] = s;
}

// Adam step on the packed parameters.
__global__ void adam_kernel(int count, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// ---------------------------------------------------------------------------
// Model object
// ---------------------------------------------------------------------------
constexpr float kLam = 0.05f, kEps = 1e-4f, kSpread = 1.0f;

static int ensure_rows(MlpModel* M, int rows)
{
    if (rows <= M->cap_rows) return KNNG_OK;
    cudaFree(M->Xb);
    cudaFree(M->A);
    cudaFree(M->Hh);
    cudaFree(M->Z);
    cudaFree(M->dZ);
    M->Xb = M->A = M->Hh = M->Z = M->dZ = nullptr;
    M->cap_rows = 0;
    if (cudaMalloc(&M->Xb, sizeof(float) * (size_t)rows * M->d) != cudaSuccess ||
        cudaMalloc(&M->A, sizeof(float) * (size_t)rows * M->H) != cudaSuccess ||
        cudaMalloc(&M->Hh, sizeof(float) * (size_t)rows * M->H) != cudaSuccess ||
        cudaMalloc(&M->Z, sizeof(float) * (size_t)rows * M->C) != cudaSuccess ||
        cudaMalloc(&M->dZ, sizeof(float) * (size_t)rows * M->C) != cudaSuccess) {
        cudaGetLastError();
        return KNNG_ERR_OOM;
    }
    M->cap_rows = rows;
    return KNNG_OK;
}

// Loss and packed gradient of the batch Xb (rows = 2B) into M->g.
static cudaError_t loss_grad(MlpModel* M, const float* Xb, int B, cudaStream_t st)
{
    const int N = 2 * B, d = M->d, H = M->H, C = M->C;
    gemm<false, true, 1>(N, H, d, Xb, d, M->W1(), d, M->Hh, H, M->b1(), M->A, st);
    gemm<false, true, 3>(N, C, H, M->Hh, H, M->W2(), H, M->Z, C, M->b2(), nullptr, st);
    const size_t lsm = sizeof(float) * (6 * C + C * C + kLossThreads);
    loss_kernel<<<1, kLossThreads, lsm, st>>>(M->Z, N, C, kLam, kEps, kSpread, M->dZ, M->loss);
    tanh_back_kernel<<<(N * C + 255) / 256, 256, 0, st>>>((int64_t)N * C, M->Z, M->dZ);
    note_launches(2);
    float* gW1 = M->g;
    float* gb1 = gW1 + (int64_t)H * d;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + (int64_t)C * H;
    gemm<true, false, 0>(C, H, N, M->dZ, C, M->Hh, H, gW2, H, nullptr, nullptr, st);  // dZ^T Hh
    colsum_kernel<<<(C + 127) / 128, 128, 0, st>>>(N, C, M->dZ, gb2);
    note_launches(1);
    gemm<false, false, 0>(N, H, C, M->dZ, C, M->W2(), H, M->Hh, H, nullptr, nullptr, st);  // dH = dZ W2 (into Hh)
    gelu_back_kernel<<<std::max(1, std::min(num_sms() * 8, (N * H + 255) / 256)), 256, 0, st>>>((int64_t)N * H,
                                                                                                  M->A, M->Hh);
    note_launches(1);
    gemm<true, false, 0>(H, d, N, M->Hh, H, Xb, d, gW1, d, nullptr, nullptr, st);  // dA^T X
    colsum_kernel<<<(H + 127) / 128, 128, 0, st>>>(N, H, M->Hh, gb1);
    note_launches(1);
    return cudaGetLastError();
}

int mlp_dims(const MlpModel* M, int* d, int* H, int* C)
{
    *d = M->d;
    *H = M->H;
    *C = M->C;
    return KNNG_OK;
}

}  // namespace knng

using namespace knng;

struct knng_mlp {
    MlpModel m;
};

extern "C" {

int knng_mlp_create(int32_t device, int32_t d_in, int32_t hidden, int32_t d_out, uint64_t seed, knng_mlp** out)
{
    if (!out) return KNNG_ERR_INVALID_ARG;
    *out = nullptr;
    if (d_in < 1 || d_in > 1024 || hidden < 16 || hidden > 256 || hidden % 16 || (d_out != 16 && d_out != 32))
        return KNNG_ERR_INVALID_ARG;
    int cnt = 0;
    if (cudaGetDeviceCount(&cnt) != cudaSuccess || device < 0 || device >= cnt) {
        cudaGetLastError();
        return KNNG_ERR_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    knng_mlp* o = new knng_mlp();
    MlpModel& M = o->m;
    M.device = device;
    M.d = d_in;
    M.H = hidden;
    M.C = d_out;
    M.count = (int64_t)hidden * d_in + hidden + (int64_t)d_out * hidden + d_out;
    std::vector<float> host(M.count, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (int64_t e = 0; e < (int64_t)hidden * d_in; ++e) host[e] = (float)(nd(rng) / std::sqrt((double)d_in));
    float* w2 = host.data() + (int64_t)hidden * d_in + hidden;
    for (int64_t e = 0; e < (int64_t)d_out * hidden; ++e) w2[e] = (float)(nd(rng) / std::sqrt((double)hidden));
    int rc = KNNG_OK;
    if (cudaMalloc(&M.w, sizeof(float) * M.count) != cudaSuccess ||
        cudaMalloc(&M.g, sizeof(float) * M.count) != cudaSuccess ||
        cudaMalloc(&M.am, sizeof(float) * M.count) != cudaSuccess ||
        cudaMalloc(&M.av, sizeof(float) * M.count) != cudaSuccess || cudaMalloc(&M.loss, sizeof(float)) != cudaSuccess)
        rc = KNNG_ERR_OOM;
    if (rc == KNNG_OK) {
        cudaMemcpy(M.w, host.data(), sizeof(float) * M.count, cudaMemcpyHostToDevice);
        cudaMemset(M.am, 0, sizeof(float) * M.count);
        cudaMemset(M.av, 0, sizeof(float) * M.count);
    }
    cudaSetDevice(prev);
    if (rc != KNNG_OK) {
        cudaGetLastError();
        knng_mlp_destroy(o);
        return rc;
    }
    *out = o;
    return KNNG_OK;
}

int knng_mlp_destroy(knng_mlp* o)
{
    if (!o) return KNNG_ERR_INVALID_ARG;
    MlpModel& M = o->m;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(M.device);
    cudaDeviceSynchronize();
    for (float* p : {M.w, M.g, M.am, M.av, M.Xb, M.A, M.Hh, M.Z, M.dZ, M.loss}) cudaFree(p);
    cudaFree(M.img);
    cudaSetDevice(prev);
    delete o;
    return KNNG_OK;
}

int knng_mlp_param_count(const knng_mlp* o, int64_t* count)
{
    if (!o || !count) return KNNG_ERR_INVALID_ARG;
    *count = o->m.count;
    return KNNG_OK;
}

int knng_mlp_get_params(const knng_mlp* o, float* host)
{
    if (!o || !host) return KNNG_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(o->m.device);
    const cudaError_t e = cudaMemcpy(host, o->m.w, sizeof(float) * o->m.count, cudaMemcpyDeviceToHost);
    cudaSetDevice(prev);
    return e == cudaSuccess ? KNNG_OK : KNNG_ERR_CUDA;
}

int knng_mlp_set_params(knng_mlp* o, const float* host)
{
    if (!o || !host) return KNNG_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(o->m.device);
    const cudaError_t e = cudaMemcpy(o->m.w, host, sizeof(float) * o->m.count, cudaMemcpyHostToDevice);
    o->m.img_stale = true;
    cudaSetDevice(prev);
    return e == cudaSuccess ? KNNG_OK : KNNG_ERR_CUDA;
}

int knng_mlp_get_adam_state(const knng_mlp* o, float* m1_host, float* m2_host, int64_t* t)
{
    if (!o || !m1_host || !m2_host || !t) return KNNG_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(o->m.device);
    cudaError_t e = cudaMemcpy(m1_host, o->m.am, sizeof(float) * o->m.count, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(m2_host, o->m.av, sizeof(float) * o->m.count, cudaMemcpyDeviceToHost);
    *t = o->m.adam_t;
    cudaSetDevice(prev);
    return e == cudaSuccess ? KNNG_OK : KNNG_ERR_CUDA;
}

int knng_mlp_set_adam_state(knng_mlp* o, const float* m1_host, const float* m2_host, int64_t t)
{
    if (!o || !m1_host || !m2_host || t < 0) return KNNG_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(o->m.device);
    cudaError_t e = cudaMemcpy(o->m.am, m1_host, sizeof(float) * o->m.count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(o->m.av, m2_host, sizeof(float) * o->m.count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) o->m.adam_t = t;
    cudaSetDevice(prev);
    return e == cudaSuccess ? KNNG_OK : KNNG_ERR_CUDA;
}

int knng_mlp_loss_grad(knng_mlp* o, const float* Xpairs, int32_t B, float* loss, float* grad, void* stream)
{
    if (!o || !Xpairs || B < 2 || !loss || !grad) return KNNG_ERR_INVALID_ARG;
    MlpModel& M = o->m;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(M.device);
    int rc = ensure_rows(&M, 2 * B);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (rc == KNNG_OK) {
        cudaError_t e = loss_grad(&M, Xpairs, B, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(grad, M.g, sizeof(float) * M.count, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(loss, M.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = KNNG_ERR_CUDA;
    }
    cudaSetDevice(prev);
    return rc;
}

int knng_mlp_train(knng_mlp* o, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ld, const int32_t* ids,
                   int32_t k, int32_t steps, int32_t batch_edges, float lr, uint64_t seed, float* last_loss,
                   void* stream)
{
    if (!o || !X || !ids || n < 2 || k < 1 || steps < 0 || batch_edges < 2 || lr <= 0.f) return KNNG_ERR_INVALID_ARG;
    if (dtype != KNNG_DTYPE_F32 && dtype != KNNG_DTYPE_F16 && dtype != KNNG_DTYPE_U8) return KNNG_ERR_INVALID_ARG;
    MlpModel& M = o->m;
    if (d != M.d || ld < d || ld >= (int64_t)1 << 31 || n >= (int64_t)1 << 31) return KNNG_ERR_INVALID_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(M.device);
    int rc = ensure_rows(&M, 2 * batch_edges);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t es = dtype == KNNG_DTYPE_F16 ? 2 : dtype == KNNG_DTYPE_U8 ? 1 : 4;
    const size_t align = dtype == KNNG_DTYPE_F16 ? 8 : dtype == KNNG_DTYPE_U8 ? 4 : 16;
    const bool vec = ((uintptr_t)X % align == 0) && ((size_t)ld * es % align == 0);
    for (int s = 0; s < steps && rc == KNNG_OK; ++s) {
        const int blocks = (batch_edges * 32 + 255) / 256;
        if (dtype == KNNG_DTYPE_F16) {
            RowLoader<kDtF16> L{X, ld, d, vec};
            sample_batch_kernel<kDtF16><<<blocks, 256, 0, st>>>(L, n, ids, k, batch_edges, seed, (uint32_t)s, M.Xb);
        } else if (dtype == KNNG_DTYPE_U8) {
            RowLoader<kDtU8> L{X, ld, d, vec};
            sample_batch_kernel<kDtU8><<<blocks, 256, 0, st>>>(L, n, ids, k, batch_edges, seed, (uint32_t)s, M.Xb);
        } else {
            RowLoader<kDtF32> L{X, ld, d, vec};
            sample_batch_kernel<kDtF32><<<blocks, 256, 0, st>>>(L, n, ids, k, batch_edges, seed, (uint32_t)s, M.Xb);
        }
        note_launches(1);
        cudaError_t e = loss_grad(&M, M.Xb, batch_edges, st);
        ++M.adam_t;
        const float c1 = 1.f - powf(0.9f, (float)M.adam_t), c2 = 1.f - powf(0.999f, (float)M.adam_t);
        adam_kernel<<<(int)((M.count + 255) / 256), 256, 0, st>>>((int)M.count, M.w, M.g, M.am, M.av, lr, 0.9f,
                                                                 0.999f, 1e-8f, c1, c2);
        note_launches(1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) rc = KNNG_ERR_CUDA;
    }
    M.img_stale = true;
    if (rc == KNNG_OK && last_loss) {
        if (cudaMemcpyAsync(last_loss, M.loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = KNNG_ERR_CUDA;
    }
    cudaSetDevice(prev);
    return rc;
}

int knng_mlp_save(const knng_mlp* o, const char* path)
{
    if (!o || !path) return KNNG_ERR_INVALID_ARG;
    std::vector<float> host(o->m.count);
    if (knng_mlp_get_params(o, host.data()) != KNNG_OK) return KNNG_ERR_CUDA;
    FILE* f = fopen(path, "wb");
    if (!f) return KNNG_ERR_INVALID_ARG;
    const int32_t hdr[4] = {0x4B4E4D31 /* "KNM1" */, o->m.d, o->m.H, o->m.C};
    const bool ok = fwrite(hdr, sizeof hdr, 1, f) == 1 && fwrite(host.data(), sizeof(float), host.size(), f) == host.size();
    fclose(f);
    return ok ? KNNG_OK : KNNG_ERR_INVALID_ARG;
}

int knng_mlp_load(knng_mlp* o, const char* path)
{
    if (!o || !path) return KNNG_ERR_INVALID_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return KNNG_ERR_INVALID_ARG;
    int32_t hdr[4];
    std::vector<float> host(o->m.count);
    bool ok = fread(hdr, sizeof hdr, 1, f) == 1 && hdr[0] == 0x4B4E4D31 && hdr[1] == o->m.d && hdr[2] == o->m.H &&
              hdr[3] == o->m.C && fread(host.data(), sizeof(float), host.size(), f) == host.size();
    fclose(f);
    if (!ok) return KNNG_ERR_INVALID_ARG;
    return knng_mlp_set_params(o, host.data());
}

}  // extern "C"

namespace knng {
MlpModel* mlp_model(knng_mlp* o) { return o ? &o->m : nullptr; }
}  // namespace knng
