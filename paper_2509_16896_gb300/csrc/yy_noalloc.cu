// yy_weighted_moments_static: weighted moments of node rows with no device allocation.
//
// This entry point exists for callers that cannot allocate device memory at the moment
// they need the result: code that runs inside a host callback or another library's
// stream work where cudaMalloc is not allowed, plug-ins whose host application owns all
// device memory and hands out only input and output buffers, and hard real-time loops
// that forbid allocation after start-up.  Such a caller cannot provide the reduction
// scratch that the handle-based API keeps in its workspace, so this variant keeps its
// scratch in a fixed array in the library's own device image instead.
//
// The scratch array below is a file-scope __device__ array of kScratchDoubles doubles
// (about 2 MB).  Every GPU that loads the library holds one copy of it until the process
// exits.  Its device address is obtained once per device with cudaGetSymbolAddress; the
// first call on each device does that set-up, so make that first call before capturing
// any stream into a CUDA graph.  All calls share the one array and it keeps whatever the
// last call left there: calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.  Nothing in
// the array has to start at zero: each call writes every slot it later reads.
#include <mutex>

#include "yy_internal.cuh"

namespace yy {
namespace noalloc {

constexpr int kBlocks = 120;                  // reduction blocks (fixed: sizes the scratch)
constexpr int kMaxDim = YY_NOALLOC_MAX_DIM;   // largest r accepted
constexpr int kDimsPerThread = kMaxDim / 256;
constexpr int kPartStride = 4 + 2 * kMaxDim;  // W, Q, (spare x2), mean[kMaxDim], M2[kMaxDim]
constexpr size_t kScratchDoubles = 2 * kBlocks + 2 + (size_t)kBlocks * kPartStride;

// Layout: [0, 2 kBlocks) log-sum-exp partials, [2 kBlocks] the merged log-sum-exp,
// [2 kBlocks + 2, ...) moment partials, kPartStride doubles per block.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

__device__ __forceinline__ void lse_merge_na(double& m, double& s, double m2, double s2) {
    if (m2 == -INFINITY) return;
    if (m == -INFINITY) { m = m2; s = s2; return; }
    if (m2 > m) { s = s * exp(m - m2) + s2; m = m2; }
    else { s += s2 * exp(m2 - m); }
}

__global__ void __launch_bounds__(256) k_na_lse(const float* __restrict__ logw, long long n, double* scr) {
    __shared__ double sm[8], ss[8];
    double m = -INFINITY, s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        lse_merge_na(m, s, (double)logw[i], 1.0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double m2 = __shfl_xor_sync(0xffffffffu, m, o);
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
        lse_merge_na(m, s, m2, s2);
    }
    if ((threadIdx.x & 31) == 0) { sm[threadIdx.x >> 5] = m; ss[threadIdx.x >> 5] = s; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double M = -INFINITY, S = 0.0;
        for (int w = 0; w < 8; ++w) lse_merge_na(M, S, sm[w], ss[w]);
        scr[2 * blockIdx.x] = M;
        scr[2 * blockIdx.x + 1] = S;
    }
}

__global__ void k_na_lse_merge(double* scr) {
    if (threadIdx.x != 0) return;
    double M = -INFINITY, S = 0.0;
    for (int b = 0; b < kBlocks; ++b) lse_merge_na(M, S, scr[2 * b], scr[2 * b + 1]);
    scr[2 * kBlocks] = (M == -INFINITY) ? -INFINITY : M + log(S);
}

// Per block: weight sum, sum of squared weights, weighted mean and centred second moment
// of the block's rows, accumulated over 32-row chunks with Chan's merge.
__global__ void __launch_bounds__(256) k_na_moments(const float* __restrict__ u, long long n, int r, long long ld,
                                                    const float* __restrict__ logw, double* scr) {
    __shared__ float w_s[32];
    __shared__ double wc_s[2];
    const int tid = threadIdx.x;
    const double lse = scr[2 * kBlocks];
    const long long rows_per = (n + gridDim.x - 1) / gridDim.x;
    const long long i0 = blockIdx.x * rows_per;
    const long long i1 = min(n, i0 + rows_per);
    double W = 0.0, Q = 0.0;
    double mu[kDimsPerThread], M2[kDimsPerThread];
#pragma unroll
    for (int q = 0; q < kDimsPerThread; ++q) { mu[q] = 0.0; M2[q] = 0.0; }
    for (long long c0 = i0; c0 < i1; c0 += 32) {
        const int cn = (int)min((long long)32, i1 - c0);
        if (tid < 32) {
            float w = 0.f;
            if (tid < cn && lse != -INFINITY) w = expf((float)((double)logw[c0 + tid] - lse));
            w_s[tid] = w;
            double a = w, b2 = (double)w * (double)w;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                b2 += __shfl_xor_sync(0xffffffffu, b2, o);
            }
            if (tid == 0) { wc_s[0] = a; wc_s[1] = b2; }
        }
        __syncthreads();
        const double Wc = wc_s[0];
        if (Wc > 0.0) {
#pragma unroll
            for (int q = 0; q < kDimsPerThread; ++q) {
                const int d = tid + 256 * q;
                if (d < r) {
                    float S = 0.f;
                    for (int l = 0; l < cn; ++l) S += w_s[l] * u[(size_t)(c0 + l) * ld + d];
                    const float muc = S / (float)Wc;
                    float m2 = 0.f;
                    for (int l = 0; l < cn; ++l) {
                        const float dv = u[(size_t)(c0 + l) * ld + d] - muc;
                        m2 += w_s[l] * dv * dv;
                    }
                    const double delta = (double)muc - mu[q];
                    const double Wn = W + Wc;
                    mu[q] += delta * (Wc / Wn);
                    M2[q] += (double)m2 + delta * delta * (W * Wc / Wn);
                }
            }
            W += Wc;
            Q += wc_s[1];
        }
        __syncthreads();
    }
    double* p = scr + 2 * kBlocks + 2 + (size_t)blockIdx.x * kPartStride;
    if (tid == 0) { p[0] = W; p[1] = Q; }
#pragma unroll
    for (int q = 0; q < kDimsPerThread; ++q) {
        const int d = tid + 256 * q;
        if (d < r) { p[4 + d] = mu[q]; p[4 + kMaxDim + d] = M2[q]; }
    }
}

// Merge of the block moments; out = mean[r], var[r], ess, lse, wsum.
__global__ void k_na_finalize(int r, const double* scr, double* __restrict__ out) {
    const double* base = scr + 2 * kBlocks + 2;
    for (int d = threadIdx.x; d < r; d += blockDim.x) {
        double W = 0.0, mu = 0.0, M2 = 0.0;
        for (int b = 0; b < kBlocks; ++b) {
            const double* p = base + (size_t)b * kPartStride;
            const double Wc = p[0];
            if (!(Wc > 0.0)) continue;
            const double delta = p[4 + d] - mu;
            const double Wn = W + Wc;
            mu += delta * (Wc / Wn);
            M2 += p[4 + kMaxDim + d] + delta * delta * (W * Wc / Wn);
            W = Wn;
        }
        out[d] = mu;
        out[r + d] = (W > 0.0) ? M2 / W : 0.0;
    }
    if (threadIdx.x == 0) {
        double W = 0.0, Q = 0.0;
        for (int b = 0; b < kBlocks; ++b) { W += base[(size_t)b * kPartStride]; Q += base[(size_t)b * kPartStride + 1]; }
        out[2 * r] = (Q > 0.0) ? W * W / Q : 0.0;
        out[2 * r + 1] = scr[2 * kBlocks];
        out[2 * r + 2] = W;
    }
}

// Device address of g_scratch, looked up once per device (with that device current).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

// Launches one kernel through cudaLaunchKernel, whose return value is the error of that
// launch alone (cudaGetLastError would also report, and clear, an error left on the thread
// by unrelated earlier work).
template <typename... Args>
cudaError_t launch_own(void (*kern)(Args...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
    void* argv[] = {static_cast<void*>(&args)...};
    return cudaLaunchKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(block), argv, 0, s);
}

}  // namespace noalloc
}  // namespace yy

extern "C" yy_status yy_weighted_moments_static(const float* d_u, int64_t n, int32_t r, int64_t ld,
                                                 const float* d_logw, double* d_out, void* stream) {
    using namespace yy::noalloc;
    if (!d_u || !d_logw || !d_out || n < 1 || r < 1 || r > kMaxDim || ld < r) return YY_ERR_ARG;
    double* scr = nullptr;
    if (scratch_for_current_device(&scr) != cudaSuccess) return YY_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const long long nn = n, lld = ld;
    const int rr = r;
    cudaError_t e = launch_own(k_na_lse, kBlocks, 256, s, d_logw, nn, scr);
    if (e == cudaSuccess) e = launch_own(k_na_lse_merge, 1, 32, s, scr);
    if (e == cudaSuccess) e = launch_own(k_na_moments, kBlocks, 256, s, d_u, nn, rr, lld, d_logw, scr);
    if (e == cudaSuccess) e = launch_own(k_na_finalize, 1, 256, s, rr, static_cast<const double*>(scr), d_out);
    return e == cudaSuccess ? YY_OK : YY_ERR_CUDA;
}
