// Restart-proposal network: a 3-layer perceptron trained and run on the GPU with the
// library's own kernels (a library addition; the paper's restart, "Local Resampling-Restart
// Mechanism", uses a fixed box at the estimate).
//
//   z = [x_hat; sqrt(v_hat); dy / sqrt(dt)] (3r), zn = clamp((z - mu) / s, -4, 4) (per-feature
//   statistics of the training set)  ->  relu(W1 zn + b1) (H)  ->  relu(W2 . + b2) (H)
//     ->  o = W3 . + b3 = [delta; lambda] (2r)
//   proposed box: centre x_hat + delta, half-widths R exp(lambda)
//   loss: mean over rows and coordinates of (t - delta)^2 / (2 sigma^2) + log sigma,
//         sigma = (R / 3) exp(lambda), t = x_true - x_hat
//
// Arithmetic: every matrix product rounds both operands to bfloat16 and accumulates in
// float32 on the tensor cores (tcgen05.mma kind::f16, accumulators in TMEM); the master
// weights, gradients and Adam moments are float32.  Kernels: the product
// C = op(A) op(B) with bias / ReLU epilogue, ReLU backward, column sums (bias
// gradients), the loss gradient, Adam, and the row gather of a training batch.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <algorithm>
#include <random>
#include <vector>

#include "yy_handle.cuh"
#include "yy_tcgen05.cuh"

using namespace yy;

struct yy_mlp {
    int r, H, max_batch;
    cudaStream_t stream;
    float* params;      // packed W1 [H][3r], b1 [H], W2 [H][H], b2 [H], W3 [2r][H], b3 [2r]
    float* grads;
    float* m;
    float* v;
    float* x;           // [max_batch][3r] gathered inputs
    float* xn;          // [max_batch][3r] normalised inputs
    float* mu;          // [3r] input normalisation: mean
    float* istd;        // [3r] input normalisation: 1 / standard deviation
    float* t;           // [max_batch][r]  gathered targets
    float* a1; float* h1; float* a2; float* h2; float* o;   // activations
    float* g_o; float* g_h; float* g_a;                     // backward scratch [max_batch][max(H, 2r)]
    float* loss;        // [1]
    int* idx;           // [max_batch] batch rows
    unsigned int* status;   // timeout bit of the tensor-core products
    long long step;
    long long n_params;
    size_t off_W1, off_b1, off_W2, off_b2, off_W3, off_b3;
};

namespace {

// ---- matrix products on the tensor cores --------------------------------------------
// C[m][n] (+)= sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn]
// (any strides, so transposed operands need no copy); epilogue: + bias[n], the
// pre-activation stored to pre (if not NULL), ReLU if relu.  One CTA of 4 warps per output
// tile of 128 rows x 64 columns: per chunk of 64 k the threads round both operands to
// bfloat16 (round to nearest even) and write them to shared memory in the K-major layout
// of the 128-byte swizzle (rows of 128 bytes, 16-byte chunk c of row r at c xor (r mod 8),
// the layout a TMA tile copy with that swizzle produces), then one thread issues four
// tcgen05.mma kind::f16 (M 128, N 64, K 16, FP32 accumulation in TMEM) and commits them to
// an mbarrier.  The epilogue warps read their 32 TMEM lanes (one output row per thread)
// with tcgen05.ld.  Rows, columns and k beyond the matrix are zero in shared memory and
// not stored.  The MMA wait is bounded (1 s): on expiry the kernel records the timeout
// bit in the network's status word, waits (bounded) for its own MMAs and frees TMEM.
constexpr int GM = 128, GN = 64, GK = 64;
constexpr uint32_t kGemmIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GN >> 3) << 17) |
                                ((uint32_t)(GM >> 4) << 24);
constexpr unsigned long long kGemmWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
    return (uint32_t)(row * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ bool gemm_wait(uint64_t* bar, uint32_t parity, unsigned long long limit) {
    if (yy::ptx::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = yy::ptx::globaltimer();
    while (!yy::ptx::mbar_try_wait(bar, parity))
        if (yy::ptx::globaltimer() - t0 > limit) return false;
    return true;
}

__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, const float* __restrict__ A, long long sam,
                                                 long long sak, const float* __restrict__ Bm, long long sbk,
                                                 long long sbn, float* __restrict__ C, long long ldc,
                                                 const float* __restrict__ bias, float* __restrict__ pre, int relu,
                                                 int accumulate, unsigned int* status) {
    using namespace yy::ptx;
    __shared__ __align__(1024) uint8_t sA[GM * GK * 2];
    __shared__ __align__(1024) uint8_t sB[GN * GK * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long m0 = (long long)blockIdx.y * GM, n0 = (long long)blockIdx.x * GN;
    if ((smem_u32(sA) | smem_u32(sB)) & 1023u) {   // the swizzle atoms need 1024-byte alignment
        if (tid == 0) atomicOr(status, kStatusNonFinite);
        return;
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        s_fail = 0;
    }
    if (warp == 0) {
        tmem_alloc(&tmem_slot, GN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const int nchunks = (K + GK - 1) / GK;
    const bool a_krow = (sak == 1);   // k contiguous in A: consecutive threads take consecutive k
    const bool b_kcol = (sbk == 1);
    bool ok = true;
    int kc_fail = 0;
    for (int kc = 0; kc < nchunks; ++kc) {
        const int k0 = kc * GK;
        for (int q = 0; q < GM * GK / 128; ++q) {
            const int e = tid + 128 * q;
            const int row = a_krow ? (e >> 6) : (e & (GM - 1));
            const int kk = a_krow ? (e & 63) : (e >> 7);
            const long long m = m0 + row, k = k0 + kk;
            const float v = (m < M && k < K) ? A[m * sam + k * sak] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(sA + sw128_offset(row, kk)) = __float2bfloat16_rn(v);
        }
        for (int q = 0; q < GN * GK / 128; ++q) {
            const int e = tid + 128 * q;
            const int col = b_kcol ? (e >> 6) : (e & (GN - 1));
            const int kk = b_kcol ? (e & 63) : (e >> 6);
            const long long n = n0 + col, k = k0 + kk;
            const float v = (n < N && k < K) ? Bm[k * sbk + n * sbn] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(sB + sw128_offset(col, kk)) = __float2bfloat16_rn(v);
        }
        // generic-proxy writes of shared memory become visible to the tensor cores' reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int kk = 0; kk < GK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), kGemmIdesc, (kc | kk) != 0 ? 1u : 0u);
            mma_commit(&bar);
        }
        // every thread waits for the chunk's MMAs before shared memory is written again
        if (!gemm_wait(&bar, (uint32_t)(kc & 1), kGemmWaitNs)) s_fail = 1;
        __syncthreads();
        tc_fence_after();
        if (s_fail) { ok = false; kc_fail = kc; break; }
    }
    if (!ok) {
        if (tid == 0) atomicOr(status, kStatusTimeout);
        gemm_wait(&bar, (uint32_t)(kc_fail & 1), kGemmWaitNs);   // our MMAs of that chunk, bounded
    } else if (nchunks > 0) {
        uint32_t v0[32], v1[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        tmem_ld32(taddr, v0);
        tmem_ld32(taddr + 32, v1);
        tmem_ld_wait();
        const long long m = m0 + warp * 32 + lane;
        if (m < M) {
#pragma unroll
            for (int c = 0; c < GN; ++c) {
                const long long n = n0 + c;
                if (n >= N) break;
                float v = __uint_as_float(c < 32 ? v0[c] : v1[c - 32]);
                if (accumulate) v += C[m * ldc + n];
                if (bias) v += bias[n];
                if (pre) pre[m * ldc + n] = v;
                if (relu) v = fmaxf(v, 0.f);
                C[m * ldc + n] = v;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, GN);
    }
}

void gemm(cudaStream_t s, unsigned int* status, int M, int N, int K, const float* A, long long sam, long long sak,
          const float* B, long long sbk, long long sbn, float* C, long long ldc, const float* bias, float* pre,
          bool relu, bool accumulate) {
    if (M < 1 || N < 1 || K < 1) return;
    dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM);
    k_gemm_tc<<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, pre, relu ? 1 : 0,
                                   accumulate ? 1 : 0, status);
}

__global__ void k_normalise(int B, int w, const float* __restrict__ x, const float* __restrict__ mu,
                            const float* __restrict__ istd, float* __restrict__ xn) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * w) return;
    const int c = i % w;
    xn[i] = fminf(fmaxf((x[i] - mu[c]) * istd[c], -4.f), 4.f);
}

__global__ void k_fill(int n, float* __restrict__ p, float v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_relu_back(int n, const float* __restrict__ g_h, const float* __restrict__ a, float* __restrict__ g_a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) g_a[i] = a[i] > 0.f ? g_h[i] : 0.f;
}

// column sums of g [M][N] into out [N]
__global__ void k_colsum(int M, int N, const float* __restrict__ g, float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += g[(size_t)m * N + n];
    out[n] = s;
}

// loss and its gradient with respect to o = [delta; lambda]
__global__ void k_loss_grad(int B, int r, const float* __restrict__ o, const float* __restrict__ t, float R,
                            float* __restrict__ g_o, float* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < B * r) {
        const int b = i / r, d = i % r;
        const float delta = o[b * 2 * r + d], lam = o[b * 2 * r + r + d];
        const float sigma = (R / 3.f) * expf(lam);
        const float e = t[b * r + d] - delta;
        const float is2 = 1.f / (sigma * sigma);
        const float sc = 1.f / (float)(B * r);
        g_o[b * 2 * r + d] = -e * is2 * sc;
        g_o[b * 2 * r + r + d] = (1.f - e * e * is2) * sc;
        l = (0.5f * e * e * is2 + logf(sigma)) * sc;
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o2);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_gather(int B, int w, const int* __restrict__ idx, const float* __restrict__ src, float* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * w) return;
    const int b = i / w, c = i % w;
    dst[i] = src[(size_t)idx[b] * w + c];
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
    size_t params, grads, m, v, x, xn, mu, istd, t, a1, h1, a2, h2, o, g_o, g_h, g_a, loss, idx, status, total;
    long long n_params;
};

Layout layout(int r, int H, int mb) {
    Layout L{};
    const long long np = (long long)H * 3 * r + H + (long long)H * H + H + 2LL * r * H + 2 * r;
    L.n_params = np;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += al256(bytes); return o; };
    L.params = take(sizeof(float) * np);
    L.grads = take(sizeof(float) * np);
    L.m = take(sizeof(float) * np);
    L.v = take(sizeof(float) * np);
    L.x = take(sizeof(float) * (size_t)mb * 3 * r);
    L.xn = take(sizeof(float) * (size_t)mb * 3 * r);
    L.mu = take(sizeof(float) * 3 * (size_t)r);
    L.istd = take(sizeof(float) * 3 * (size_t)r);
    L.t = take(sizeof(float) * (size_t)mb * r);
    L.a1 = take(sizeof(float) * (size_t)mb * H);
    L.h1 = take(sizeof(float) * (size_t)mb * H);
    L.a2 = take(sizeof(float) * (size_t)mb * H);
    L.h2 = take(sizeof(float) * (size_t)mb * H);
    L.o = take(sizeof(float) * (size_t)mb * 2 * r);
    const int wmax = H > 2 * r ? H : 2 * r;
    L.g_o = take(sizeof(float) * (size_t)mb * 2 * r);
    L.g_h = take(sizeof(float) * (size_t)mb * wmax);
    L.g_a = take(sizeof(float) * (size_t)mb * wmax);
    L.loss = take(sizeof(float));
    L.idx = take(sizeof(int) * (size_t)mb);
    L.status = take(sizeof(unsigned int));
    L.total = off + 256;
    return L;
}

void forward(yy_mlp* n, const float* x, int B) {
    const int r = n->r, H = n->H;
    const float* P = n->params;
    k_normalise<<<(B * 3 * r + 255) / 256, 256, 0, n->stream>>>(B, 3 * r, x, n->mu, n->istd, n->xn);
    gemm(n->stream, n->status, B, H, 3 * r, n->xn, 3 * r, 1, P + n->off_W1, 1, 3 * r, n->h1, H, P + n->off_b1, n->a1, true, false);
    gemm(n->stream, n->status, B, H, H, n->h1, H, 1, P + n->off_W2, 1, H, n->h2, H, P + n->off_b2, n->a2, true, false);
    gemm(n->stream, n->status, B, 2 * r, H, n->h2, H, 1, P + n->off_W3, 1, H, n->o, 2 * r, P + n->off_b3, nullptr, false, false);
}

// forward + backward on the gathered batch (n->x, n->t); gradients into n->grads, loss into n->loss
void forward_backward(yy_mlp* n, int B, float R) {
    const int r = n->r, H = n->H;
    const float* P = n->params;
    float* G = n->grads;
    cudaStream_t s = n->stream;
    forward(n, n->x, B);
    cudaMemsetAsync(n->loss, 0, sizeof(float), s);
    k_loss_grad<<<(B * r + 255) / 256, 256, 0, s>>>(B, r, n->o, n->t, R, n->g_o, n->loss);
    // layer 3: g_W3 = g_o^T h2 ; g_b3 = colsum(g_o) ; g_h2 = g_o W3
    gemm(s, n->status, 2 * r, H, B, n->g_o, 1, 2 * r, n->h2, H, 1, G + n->off_W3, H, nullptr, nullptr, false, false);
    k_colsum<<<(2 * r + 127) / 128, 128, 0, s>>>(B, 2 * r, n->g_o, G + n->off_b3);
    gemm(s, n->status, B, H, 2 * r, n->g_o, 2 * r, 1, P + n->off_W3, H, 1, n->g_h, H, nullptr, nullptr, false, false);
    k_relu_back<<<(B * H + 255) / 256, 256, 0, s>>>(B * H, n->g_h, n->a2, n->g_a);
    // layer 2
    gemm(s, n->status, H, H, B, n->g_a, 1, H, n->h1, H, 1, G + n->off_W2, H, nullptr, nullptr, false, false);
    k_colsum<<<(H + 127) / 128, 128, 0, s>>>(B, H, n->g_a, G + n->off_b2);
    gemm(s, n->status, B, H, H, n->g_a, H, 1, P + n->off_W2, H, 1, n->g_h, H, nullptr, nullptr, false, false);
    k_relu_back<<<(B * H + 255) / 256, 256, 0, s>>>(B * H, n->g_h, n->a1, n->g_a);
    // layer 1
    gemm(s, n->status, H, 3 * r, B, n->g_a, 1, H, n->xn, 3 * r, 1, G + n->off_W1, 3 * r, nullptr, nullptr, false, false);
    k_colsum<<<(H + 127) / 128, 128, 0, s>>>(B, H, n->g_a, G + n->off_b1);
}

}  // namespace

// ---- restart-box proposal inside the filter (used by yy_restart with the learned rule) ----
namespace yy {

// features of one step: [x_hat - c; sqrt(v_hat); dy / sqrt(dt)] as float32, c the centre of
// the box the estimate was computed in
__global__ void k_mlp_features(int r, const double* __restrict__ mean, const double* __restrict__ var,
                               const double* __restrict__ dy, const double* __restrict__ centre, double dt,
                               const int* __restrict__ flag, float* __restrict__ z) {
    if (flag && *flag == 0) return;
    for (int d = threadIdx.x; d < r; d += blockDim.x) {
        z[d] = (float)(mean[d] - centre[d]);
        z[r + d] = (float)sqrt(fmax(var[d], 0.0));
        z[2 * r + d] = (float)(dy[d] / sqrt(dt));
    }
}

cudaError_t mlp_propose(struct ::yy_mlp* net, int r, const double* mean, const double* var, const double* dy,
                        const double* centre, double dt, const int* flag, cudaStream_t s, int* launches) {
    if (!net || net->r != r) return cudaErrorInvalidValue;
    cudaStream_t old = net->stream;
    net->stream = s;
    k_mlp_features<<<1, 256, 0, s>>>(r, mean, var, dy, centre, dt, flag, net->x);
    forward(net, net->x, 1);
    net->stream = old;
    if (launches) *launches += 5;
    return cudaGetLastError();
}

const float* mlp_output(const struct ::yy_mlp* net) { return net->o; }

}  // namespace yy

extern "C" {

int64_t yy_mlp_param_count(int32_t r, int32_t hidden) {
    if (r < 1 || r > YY_MAX_DIM || hidden < 1 || hidden > 4096) return 0;
    return layout(r, hidden, 1).n_params;
}

size_t yy_mlp_workspace_bytes(int32_t r, int32_t hidden, int32_t max_batch) {
    if (yy_mlp_param_count(r, hidden) == 0 || max_batch < 1 || max_batch > (1 << 20)) return 0;
    return layout(r, hidden, max_batch).total;
}

yy_status yy_mlp_create(int32_t r, int32_t hidden, int32_t max_batch, void* d_ws, size_t bytes, void* stream,
                        yy_mlp** out) {
    if (!out) return YY_ERR_ARG;
    *out = nullptr;
    const size_t need = yy_mlp_workspace_bytes(r, hidden, max_batch);
    if (need == 0) return YY_ERR_ARG;
    if (!d_ws || ((uintptr_t)d_ws & 255u) || bytes < need) return YY_ERR_WORKSPACE;
    yy_mlp* n = new (std::nothrow) yy_mlp();
    if (!n) return YY_ERR_ARG;
    const Layout L = layout(r, hidden, max_batch);
    char* b = (char*)d_ws;
    n->r = r; n->H = hidden; n->max_batch = max_batch;
    n->stream = (cudaStream_t)stream;
    n->params = (float*)(b + L.params); n->grads = (float*)(b + L.grads);
    n->m = (float*)(b + L.m); n->v = (float*)(b + L.v);
    n->x = (float*)(b + L.x); n->t = (float*)(b + L.t);
    n->xn = (float*)(b + L.xn); n->mu = (float*)(b + L.mu); n->istd = (float*)(b + L.istd);
    n->a1 = (float*)(b + L.a1); n->h1 = (float*)(b + L.h1); n->a2 = (float*)(b + L.a2); n->h2 = (float*)(b + L.h2);
    n->o = (float*)(b + L.o); n->g_o = (float*)(b + L.g_o); n->g_h = (float*)(b + L.g_h); n->g_a = (float*)(b + L.g_a);
    n->loss = (float*)(b + L.loss); n->idx = (int*)(b + L.idx);
    n->status = (unsigned int*)(b + L.status);
    n->n_params = L.n_params;
    n->off_W1 = 0;
    n->off_b1 = n->off_W1 + (size_t)hidden * 3 * r;
    n->off_W2 = n->off_b1 + hidden;
    n->off_b2 = n->off_W2 + (size_t)hidden * hidden;
    n->off_W3 = n->off_b2 + hidden;
    n->off_b3 = n->off_W3 + (size_t)2 * r * hidden;
    if (cudaMemsetAsync(d_ws, 0, need, n->stream) != cudaSuccess) { delete n; return YY_ERR_CUDA; }
    k_fill<<<(3 * r + 255) / 256, 256, 0, n->stream>>>(3 * r, n->istd, 1.0f);   // identity normalisation
    *out = n;
    return YY_OK;
}

yy_status yy_mlp_destroy(yy_mlp* n) {
    delete n;
    return YY_OK;
}

yy_status yy_mlp_set_params(yy_mlp* n, const float* h_params) {
    if (!n || !h_params) return YY_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(n->params, h_params, sizeof(float) * n->n_params, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, sizeof(float) * n->n_params, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, sizeof(float) * n->n_params, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    n->step = 0;
    return e == cudaSuccess ? YY_OK : YY_ERR_CUDA;
}

yy_status yy_mlp_set_input_norm(yy_mlp* n, const float* h_mean, const float* h_std) {
    if (!n || !h_mean || !h_std) return YY_ERR_ARG;
    std::vector<float> istd(3 * (size_t)n->r);
    for (int i = 0; i < 3 * n->r; ++i) {
        if (!(h_std[i] > 0.f) || !isfinite(h_mean[i])) return YY_ERR_ARG;
        istd[i] = 1.f / h_std[i];
    }
    cudaError_t e = cudaMemcpyAsync(n->mu, h_mean, sizeof(float) * 3 * n->r, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->istd, istd.data(), sizeof(float) * 3 * n->r, cudaMemcpyHostToDevice, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? YY_OK : YY_ERR_CUDA;
}

yy_status yy_mlp_get_params(yy_mlp* n, float* h_params) {
    if (!n || !h_params) return YY_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(h_params, n->params, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? YY_OK : YY_ERR_CUDA;
}

yy_status yy_mlp_forward(yy_mlp* n, const float* d_x, int32_t B, float* d_out) {
    if (!n || !d_x || !d_out || B < 1) return YY_ERR_ARG;
    const int chunk = n->max_batch;
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int bb = std::min(chunk, B - b0);
        forward(n, d_x + (size_t)b0 * 3 * n->r, bb);
        if (cudaMemcpyAsync(d_out + (size_t)b0 * 2 * n->r, n->o, sizeof(float) * bb * 2 * n->r,
                            cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess)
            return YY_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? YY_OK : YY_ERR_CUDA;
}

yy_status yy_mlp_loss_grad(yy_mlp* n, const float* d_x, const float* d_t, int32_t B, double R, float* h_loss,
                           float* h_grads) {
    if (!n || !d_x || !d_t || B < 1 || B > n->max_batch || !(R > 0.0)) return YY_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(n->x, d_x, sizeof(float) * B * 3 * n->r, cudaMemcpyDeviceToDevice, n->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n->t, d_t, sizeof(float) * B * n->r, cudaMemcpyDeviceToDevice, n->stream);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    forward_backward(n, B, (float)R);
    if (h_loss) e = cudaMemcpyAsync(h_loss, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess && h_grads)
        e = cudaMemcpyAsync(h_grads, n->grads, sizeof(float) * n->n_params, cudaMemcpyDeviceToHost, n->stream);
    unsigned int st = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, n->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    if (st & kStatusTimeout) return YY_ERR_TIMEOUT;
    return (st & kStatusNonFinite) ? YY_ERR_CUDA : YY_OK;
}

yy_status yy_mlp_train(yy_mlp* n, const float* d_x, const float* d_t, int64_t M, double R, int32_t epochs,
                       int32_t batch, float lr, uint64_t seed, float* h_last_loss) {
    if (!n || !d_x || !d_t || M < 1 || epochs < 1 || batch < 1 || batch > n->max_batch || !(R > 0.0) || !(lr > 0.f))
        return YY_ERR_ARG;
    std::mt19937_64 rng(seed);
    std::vector<int> perm((size_t)M);
    for (int64_t i = 0; i < M; ++i) perm[(size_t)i] = (int)i;
    float last = 0.f;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        for (int64_t b0 = 0; b0 + batch <= M || (b0 == 0 && M < batch); b0 += batch) {
            const int bb = (int)std::min<int64_t>(batch, M - b0);
            if (cudaMemcpyAsync(n->idx, perm.data() + b0, sizeof(int) * bb, cudaMemcpyHostToDevice, n->stream) != cudaSuccess)
                return YY_ERR_CUDA;
            k_gather<<<(bb * 3 * n->r + 255) / 256, 256, 0, n->stream>>>(bb, 3 * n->r, n->idx, d_x, n->x);
            k_gather<<<(bb * n->r + 255) / 256, 256, 0, n->stream>>>(bb, n->r, n->idx, d_t, n->t);
            forward_backward(n, bb, (float)R);
            n->step += 1;
            const float c1 = 1.f - powf(0.9f, (float)n->step), c2 = 1.f - powf(0.999f, (float)n->step);
            k_adam<<<(unsigned)((n->n_params + 255) / 256), 256, 0, n->stream>>>(n->n_params, n->params, n->grads, n->m,
                                                                               n->v, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
            // the host index buffer must stay valid until the copy has happened
            if (cudaStreamSynchronize(n->stream) != cudaSuccess) return YY_ERR_CUDA;
            if (M < batch) break;
        }
    }
    unsigned int st = 0;
    if (cudaMemcpyAsync(&last, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaMemcpyAsync(&st, n->status, sizeof(unsigned int), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
        return YY_ERR_CUDA;
    if (h_last_loss) *h_last_loss = last;
    if (st & kStatusTimeout) return YY_ERR_TIMEOUT;
    return (st & kStatusNonFinite) ? YY_ERR_CUDA : YY_OK;
}

}  // extern "C"
