// Restart-proposal network: a 3-layer perceptron trained and run on the GPU with the
// library's own kernels (a library addition; the paper's restart, Section 5, uses a fixed
// box at the estimate).
//
//   z = [x_hat; sqrt(v_hat); dy / sqrt(dt)] (3r), zn = clamp((z - mu) / s, -4, 4) (per-feature
//   statistics of the training set)  ->  relu(W1 zn + b1) (H)  ->  relu(W2 . + b2) (H)
//     ->  o = W3 . + b3 = [delta; lambda] (2r)
//   proposed box: centre x_hat + delta, half-widths R exp(lambda)
//   loss: mean over rows and coordinates of (t - delta)^2 / (2 sigma^2) + log sigma,
//         sigma = (R / 3) exp(lambda), t = x_true - x_hat
//
// Arithmetic: every matrix product rounds both operands to bfloat16 on load and
// accumulates in float32 (BF16 weights and activations, FP32 accumulation); the master
// weights, gradients and Adam moments are float32.  Kernels: a tiled product
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
    long long step;
    long long n_params;
    size_t off_W1, off_b1, off_W2, off_b2, off_W3, off_b3;
};

namespace {

constexpr int TILE = 32;

// C[m][n] (+)= sum_k A(m, k) B(k, n), A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn];
// operands rounded to bfloat16, float32 accumulation; epilogue: + bias[n], store the
// pre-activation to pre (if not NULL), ReLU if relu.
__global__ void __launch_bounds__(256) k_gemm_bf16(int M, int N, int K, const float* __restrict__ A, long long sam,
                                                   long long sak, const float* __restrict__ Bm, long long sbk,
                                                   long long sbn, float* __restrict__ C, long long ldc,
                                                   const float* __restrict__ bias, float* __restrict__ pre, int relu,
                                                   int accumulate) {
    __shared__ float As[TILE][TILE + 1], Bs[TILE][TILE + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads, 4 rows each
    const int m0 = blockIdx.y * TILE, n0 = blockIdx.x * TILE;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += TILE) {
        for (int q = 0; q < 4; ++q) {
            const int mm = ty * 4 + q;
            const int m = m0 + mm, k = k0 + tx;
            As[mm][tx] = (m < M && k < K) ? __bfloat162float(__float2bfloat16_rn(A[m * sam + k * sak])) : 0.f;
            const int kk = k0 + mm, n = n0 + tx;
            Bs[mm][tx] = (kk < K && n < N) ? __bfloat162float(__float2bfloat16_rn(Bm[kk * sbk + n * sbn])) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < TILE; ++kk) {
            const float b = Bs[kk][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(As[ty * 4 + q][kk], b, acc[q]);
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        const int m = m0 + ty * 4 + q, n = n0 + tx;
        if (m >= M || n >= N) continue;
        float v = acc[q];
        if (accumulate) v += C[m * ldc + n];
        if (bias) v += bias[n];
        if (pre) pre[m * ldc + n] = v;
        if (relu) v = fmaxf(v, 0.f);
        C[m * ldc + n] = v;
    }
}

void gemm(cudaStream_t s, int M, int N, int K, const float* A, long long sam, long long sak, const float* B,
          long long sbk, long long sbn, float* C, long long ldc, const float* bias, float* pre, bool relu,
          bool accumulate) {
    dim3 grid((N + TILE - 1) / TILE, (M + TILE - 1) / TILE);
    k_gemm_bf16<<<grid, 256, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, pre, relu ? 1 : 0,
                                      accumulate ? 1 : 0);
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
    size_t params, grads, m, v, x, xn, mu, istd, t, a1, h1, a2, h2, o, g_o, g_h, g_a, loss, idx, total;
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
    L.total = off + 256;
    return L;
}

void forward(yy_mlp* n, const float* x, int B) {
    const int r = n->r, H = n->H;
    const float* P = n->params;
    k_normalise<<<(B * 3 * r + 255) / 256, 256, 0, n->stream>>>(B, 3 * r, x, n->mu, n->istd, n->xn);
    gemm(n->stream, B, H, 3 * r, n->xn, 3 * r, 1, P + n->off_W1, 1, 3 * r, n->h1, H, P + n->off_b1, n->a1, true, false);
    gemm(n->stream, B, H, H, n->h1, H, 1, P + n->off_W2, 1, H, n->h2, H, P + n->off_b2, n->a2, true, false);
    gemm(n->stream, B, 2 * r, H, n->h2, H, 1, P + n->off_W3, 1, H, n->o, 2 * r, P + n->off_b3, nullptr, false, false);
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
    gemm(s, 2 * r, H, B, n->g_o, 1, 2 * r, n->h2, H, 1, G + n->off_W3, H, nullptr, nullptr, false, false);
    k_colsum<<<(2 * r + 127) / 128, 128, 0, s>>>(B, 2 * r, n->g_o, G + n->off_b3);
    gemm(s, B, H, 2 * r, n->g_o, 2 * r, 1, P + n->off_W3, H, 1, n->g_h, H, nullptr, nullptr, false, false);
    k_relu_back<<<(B * H + 255) / 256, 256, 0, s>>>(B * H, n->g_h, n->a2, n->g_a);
    // layer 2
    gemm(s, H, H, B, n->g_a, 1, H, n->h1, H, 1, G + n->off_W2, H, nullptr, nullptr, false, false);
    k_colsum<<<(H + 127) / 128, 128, 0, s>>>(B, H, n->g_a, G + n->off_b2);
    gemm(s, B, H, H, n->g_a, H, 1, P + n->off_W2, H, 1, n->g_h, H, nullptr, nullptr, false, false);
    k_relu_back<<<(B * H + 255) / 256, 256, 0, s>>>(B * H, n->g_h, n->a1, n->g_a);
    // layer 1
    gemm(s, H, 3 * r, B, n->g_a, 1, H, n->xn, 3 * r, 1, G + n->off_W1, 3 * r, nullptr, nullptr, false, false);
    k_colsum<<<(H + 127) / 128, 128, 0, s>>>(B, H, n->g_a, G + n->off_b1);
}

}  // namespace

// ---- restart-box proposal inside the filter (used by yy_restart with the learned rule) ----
namespace yy {

// features of one step: [x_hat; sqrt(v_hat); dy / sqrt(dt)] as float32
__global__ void k_mlp_features(int r, const double* __restrict__ mean, const double* __restrict__ var,
                               const double* __restrict__ dy, double dt, const int* __restrict__ flag,
                               float* __restrict__ z) {
    if (flag && *flag == 0) return;
    for (int d = threadIdx.x; d < r; d += blockDim.x) {
        z[d] = (float)mean[d];
        z[r + d] = (float)sqrt(fmax(var[d], 0.0));
        z[2 * r + d] = (float)(dy[d] / sqrt(dt));
    }
}

cudaError_t mlp_propose(struct ::yy_mlp* net, int r, const double* mean, const double* var, const double* dy,
                        double dt, const int* flag, cudaStream_t s, int* launches) {
    if (!net || net->r != r) return cudaErrorInvalidValue;
    cudaStream_t old = net->stream;
    net->stream = s;
    k_mlp_features<<<1, 256, 0, s>>>(r, mean, var, dy, dt, flag, net->x);
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
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    return e == cudaSuccess ? YY_OK : YY_ERR_CUDA;
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
    if (cudaMemcpyAsync(&last, n->loss, sizeof(float), cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
        cudaStreamSynchronize(n->stream) != cudaSuccess)
        return YY_ERR_CUDA;
    if (h_last_loss) *h_last_loss = last;
    return YY_OK;
}

}  // extern "C"
