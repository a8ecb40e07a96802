// Per-node preparation: drift, divergence and norms at x = c + u, Dirichlet mask, bf16
// copy of u, and the initial or restart log-weights.
//
//   f(x)      cubic: cos x (componentwise); linear: a x  ("Large-Scale Scalability Test",
//             "Linear Filtering Benchmark");
//             large-scale test: sin(x) (A x) + sin(2x) (A1 x), A and A1 upper bidiagonal
//   div f(x)  cubic: -sum_d sin x_d;       linear: a r;
//             large-scale test: sum_d cos(x_d)(A x)_d - 0.5 sin x_d + 2 cos(2 x_d)(A1 x)_d - 0.3 sin 2x_d
//   mask      |u_d| >= R_d - 1e-12 R_d for some d, tested in float64 ("Algorithm for
//             Kolmogorov Equation", step 3)
//   prior     log sigma_0(x) = -|x - mu0|^2 / (2 s0^2) + const (same algorithm, step 4)
//   restart   log N(x; x_hat, diag(max(v_hat, (R/4)^2))) + const, or uniform
//             ("Local Resampling-Restart Mechanism"; the density is this library's reading
//             of "re-initialise")
// Constants that cancel in the normalisation that follows are dropped.
//
// One warp per node row; lane l holds float2 l + 32 q of the row for q = 0 .. r_pad / 64 - 1
// (coordinates 64 q + 2 l, +1: chunk q of 64 coordinates), the whole row loaded before any
// arithmetic.  x = c + u is formed as c_hi + (u + c_lo) with the float64 centre split into a
// head and a tail in the working precision T (k_prep_dims).  In float32 the cubic drift
// comes from the angle-addition form of yy_drift.cuh; in float64 from sincos.
#include "yy_internal.cuh"
#include "yy_drift.cuh"
#include "yy_prep_dims.cuh"

#include <cuda_fp8.h>

#include <type_traits>

namespace yy {

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int kRowQ = YY_MAX_DIM / 64;   // float2 per lane of the longest row

// Drift component d of the large-scale test's model at x_d with neighbour x_{d+1} (nb = 0
// for the last coordinate: the bidiagonal matrices have no entry there), and the
// coordinate's term of div f.
__device__ __forceinline__ void e1_drift(float x, float nb, float* f, float* dv) {
    const float ax = fmaf(-0.5f, x, 0.1f * nb), a1x = fmaf(-0.3f, x, 0.3f * nb);
    float s1, c1, s2, c2;
    sincosf(x, &s1, &c1);
    sincosf(2.0f * x, &s2, &c2);
    *f = fmaf(s1, ax, s2 * a1x);
    *dv = c1 * ax - 0.5f * s1 + 2.0f * c2 * a1x - 0.3f * s2;
}
__device__ __forceinline__ void e1_drift(double x, double nb, double* f, double* dv) {
    const double ax = fma(-0.5, x, 0.1 * nb), a1x = fma(-0.3, x, 0.3 * nb);
    double s1, c1, s2, c2;
    sincos(x, &s1, &c1);
    sincos(2.0 * x, &s2, &c2);
    *f = fma(s1, ax, s2 * a1x);
    *dv = c1 * ax - 0.5 * s1 + 2.0 * c2 * a1x - 0.3 * s2;
}

template <typename T> __device__ __forceinline__ T sin_w(T x);
template <> __device__ __forceinline__ float sin_w<float>(float x) { return sinf(x); }
template <> __device__ __forceinline__ double sin_w<double>(double x) { return sin(x); }
template <typename T> __device__ __forceinline__ T log_w(T x);
template <> __device__ __forceinline__ float log_w<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double log_w<double>(double x) { return log(x); }

template <typename T>
__device__ __forceinline__ T exp_w(T x);
template <>
__device__ __forceinline__ float exp_w<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_w<double>(double x) { return exp(x); }

// The pass proper, compiled per mode and per "first" (node-only quantities too), so that
// the restart pass carries none of the other modes' float64 arithmetic.
template <typename T, int mode, bool first, bool narrow>
__device__ __forceinline__ void prep_rows(const Consts<T>& k, const Bufs<T>& b, double prior_mean,
                                          double prior_var, int bid, int nblk, const T* s_hi, const T* s_lo,
                                          const T* s_iv, const T* s_cc, const T* s_sc, T& lse_m,
                                          T& lse_s) {
    const int rp = k.r_pad;
    const int lane = threadIdx.x & 31;
    const long long warp = (bid * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)nblk * blockDim.x) >> 5;
    const double* cen = (mode == kPrepRestart) ? b.next_centre : b.centre;
    const double* halfw = (mode == kPrepRestart) ? b.next_half : b.halfwidth;
    const int nq = rp >> 6;   // float2 per lane
    const bool cubic = k.model == YY_MODEL_CUBIC;
    const bool e1 = k.model == YY_MODEL_PAPER_E1;
    for (long long i = warp; i < k.n_pad; i += nwarps) {
        const float* ui = b.u + (size_t)i * rp;
        T* fi = b.f + (size_t)i * rp;
        if (i >= k.n) {  // padding rows: inert
            if (b.store_f)
                for (int d = lane; d < rp; d += 32) fi[d] = T(0);
            if (lane == 0) {
                b.divf[i] = T(0);
                b.nf[i] = T(0);
                b.logw[i] = T(-INFINITY);
                if (b.hld) b.hld[i] = T(0);
                if (first) { b.nu[i] = T(0); b.mask[i] = 1; }
            }
            if (b.minv)
                for (int d = lane; d < rp; d += 32) b.minv[(size_t)i * rp + d] = T(0);
            if (first && b.nu_chunk)
                for (int c = lane; c < nq; c += 32) b.nu_chunk[(size_t)i * nq + c] = 0.f;
            continue;
        }
        // the whole row first: up to kRowQ loads in flight per lane
        const float2* ui2 = reinterpret_cast<const float2*>(ui);
        float2 uu[kRowQ];
#pragma unroll
        for (int q = 0; q < kRowQ; ++q) uu[q] = (q < nq) ? ui2[lane + 32 * q] : make_float2(0.f, 0.f);
        // the stored boundary mask, loaded with the row rather than after its reductions
        const uint8_t mk = first ? (uint8_t)0 : b.mask[i];
        T div = T(0), nf = T(0), nu = T(0), lw = T(0);
        T hl = T(0);   // noise coefficients: 1/2 log det_+ a(x) = sum of log U_d over U_d > 0
        int on_face = 0;
        bool done = false;
        if constexpr (std::is_same<T, float>::value && narrow && !first) {
            // the common restart and re-preparation case: cubic drift by the polynomials,
            // padded coordinates inert by construction (u = 0, cos c = sin c = 0, no Gaussian
            // term), so no per-element tests; per-dimension constants as float2 pairs
            if (cubic && k.noise == YY_NOISE_UNIT) {
#pragma unroll
                for (int q = 0; q < kRowQ; ++q) {
                    if (q >= nq) break;   // uniform over the warp
                    const int d = 64 * q + 2 * lane;
                    const float2 cc = *reinterpret_cast<const float2*>(s_cc + d);
                    const float2 sc = *reinterpret_cast<const float2*>(s_sc + d);
                    float2 f2, s2;   // both coordinates in packed pairs (same values as one by one)
                    cubic_drift_narrow2(uu[q], cc, sc, &f2, &s2);
                    const float f0 = f2.x, f1 = f2.y;
                    div -= s2.x + s2.y;
                    nf = fmaf(f0, f0, fmaf(f1, f1, nf));
                    if constexpr (mode == kPrepRestart) {
                        const float2 iv = *reinterpret_cast<const float2*>(s_iv + d);
                        lw = fmaf(-uu[q].x * uu[q].x, iv.x, fmaf(-uu[q].y * uu[q].y, iv.y, lw));
                    }
                    if (b.store_f) *reinterpret_cast<float2*>(fi + d) = make_float2(f0, f1);
                }
                done = true;
            }
        }
#pragma unroll
        for (int q = 0; q < kRowQ; ++q) {
            if (done) break;
            if (q >= nq) break;   // uniform over the warp
            const int dq = 64 * q + 2 * lane;
            float cq = 0.f;       // |u|^2 of this lane's two coordinates
            // large-scale model: u of coordinate dq + 2 (the next lane's first, or for the last
            // lane the first lane's of the next chunk; zero padding beyond the row)
            float u_next = 0.f;
            if (e1) {
                const float from_lane = __shfl_down_sync(0xffffffffu, uu[q].x, 1);
                const float from_next = __shfl_sync(0xffffffffu, (q + 1 < kRowQ) ? uu[q + 1 < kRowQ ? q + 1 : q].x : 0.f, 0);
                u_next = (lane < 31) ? from_lane : ((q + 1 < nq) ? from_next : 0.f);
            }
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int d = dq + e;
                const float uf = e ? uu[q].y : uu[q].x;
                T fv = T(0);
                if (d < k.r) {
                    if (e1) {
                        const float un = e ? u_next : uu[q].y;   // u of coordinate d + 1
                        const T x = s_hi[d] + ((T)uf + s_lo[d]);
                        const T xn = (d + 1 < k.r) ? s_hi[d + 1] + ((T)un + s_lo[d + 1]) : T(0);
                        T dv;
                        e1_drift(x, xn, &fv, &dv);
                        div += dv;
                    } else if (cubic) {
                        T sn;
                        if constexpr (std::is_same<T, float>::value && narrow) {
                            cubic_drift_narrow(uf, s_cc[d], s_sc[d], &fv, &sn);
                        } else if constexpr (std::is_same<T, float>::value) {
                            cubic_drift(uf, s_hi[d], s_lo[d], s_cc[d], s_sc[d], &fv, &sn);
                        } else {
                            sincos(s_hi[d] + ((T)uf + s_lo[d]), &sn, &fv);
                        }
                        div -= sn;
                    } else {
                        fv = k.model_a * (s_hi[d] + ((T)uf + s_lo[d]));
                        div += k.model_a;
                    }
                    // noise coefficients: |f|^2 in the metric a(x)^+ of this node, stored per
                    // coordinate for the kernel sum
                    T mval = T(1);
                    if (k.noise == YY_NOISE_DIAG) {
                        const T x = s_hi[d] + ((T)uf + s_lo[d]);
                        const T sx = sin_w<T>(x);
                        const T U = (d < k.noise_u_zero) ? T(0) : k.nz_u * (T(1) + k.nz_uk * sx * sx);
                        mval = (U > T(0)) ? T(1) / (U * U) : T(0);
                        if (U > T(0)) hl += log_w<T>(U);
                        b.minv[(size_t)i * rp + d] = mval;
                    }
                    nf += mval * fv * fv;
                    if constexpr (mode == kPrepRestart) lw -= (T)uf * (T)uf * s_iv[d];
                    if constexpr (first) {
                        nu += (T)uf * (T)uf;
                        cq = fmaf(uf, uf, cq);
                        const double R = halfw[d];
                        if (fabs((double)uf) >= R - 1e-12 * R) on_face = 1;
                    }
                    if constexpr (mode == kPrepInit) {
                        const double z = cen[d] + (double)uf - prior_mean;
                        lw -= (T)(0.5 * z * z / prior_var);
                    }
                }
                if (first && b.ubf) {
                    if (k.tc_fp8)   // e4m3 copy of s u, rows of tc_r8 bytes (tail bytes stay zero)
                        reinterpret_cast<uint8_t*>(b.ubf)[(size_t)i * k.tc_r8 + d] = (uint8_t)__nv_cvt_float_to_fp8(
                            d < k.r ? k.tc_s * uf : 0.0f, __NV_SATFINITE, __NV_E4M3);
                    else
                        b.ubf[(size_t)i * rp + d] = __float2bfloat16_rn(d < k.r ? uf : 0.0f);
                }
                if (b.store_f) fi[d] = fv;
                if (d >= k.r && b.minv) b.minv[(size_t)i * rp + d] = T(0);
            }
            if (first && b.nu_chunk) {
                cq = warp_sum(cq);
                if (lane == 0) b.nu_chunk[(size_t)i * nq + q] = cq;
            }
        }
        div = warp_sum(div);
        nf = warp_sum(nf);
        lw = warp_sum(lw);
        if (b.hld) {
            hl = warp_sum(hl);
            if (lane == 0) b.hld[i] = hl;
        }
        if (first) {
            nu = warp_sum(nu);
            on_face = __any_sync(0xffffffffu, on_face);
        }
        if (lane == 0) {
            b.divf[i] = div;
            b.nf[i] = nf;
            if (first) {
                b.nu[i] = nu;
                b.mask[i] = (uint8_t)on_face;
            }
            if (mode != kPrepOnly) {
                const bool masked = first ? (on_face != 0) : (mk != 0);
                const T out = masked ? T(-INFINITY) : lw;
                b.logw[i] = out;
                // running (max, sum) of the written log-weights (lane 0 of every warp), in the
                // working precision: float64 issue time per row is large on this part
                if (out != T(-INFINITY)) {
                    if (out > lse_m) {
                        lse_s = (lse_m == T(-INFINITY)) ? T(1) : lse_s * exp_w<T>(lse_m - out) + T(1);
                        lse_m = out;
                    } else {
                        lse_s += exp_w<T>(out - lse_m);
                    }
                }
            }
        }
    }
}

// lse_out: also write the block's (max, sum) log-sum-exp partial of the new log-weights to
// b.part[2 bid], b.part[2 bid + 1] (restart and init passes).
template <typename T>
__device__ __forceinline__ void prep_body(const Consts<T>& k, const Bufs<T>& b, int mode, int first,
                                          double prior_mean, double prior_var, int bid, int nblk, bool lse_out) {
    if (mode == kPrepRestart && b.stats->restart_flag == 0) return;
    // a restart that re-mapped the nodes to new half-widths also redoes the node-only
    // quantities (|u|^2, mask against the new faces, bf16 copy)
    if (mode == kPrepRestart && b.stats->scale_changed) first = 1;
    __shared__ T s_hi[YY_MAX_DIM], s_lo[YY_MAX_DIM], s_iv[YY_MAX_DIM], s_cc[YY_MAX_DIM], s_sc[YY_MAX_DIM];
    const int rp = k.r_pad;
    for (int d = threadIdx.x; d < rp; d += blockDim.x) {
        s_hi[d] = b.dimc[d];
        s_lo[d] = b.dimc[rp + d];
        s_iv[d] = b.dimc[2 * rp + d];
        s_cc[d] = b.dimc[3 * rp + d];
        s_sc[d] = b.dimc[4 * rp + d];
    }
    // every dimension inside the polynomials' range: no per-element fallback test
    int my_narrow = 1;
    for (int d = threadIdx.x; d < k.r; d += blockDim.x) my_narrow &= (s_cc[d] == s_cc[d]) ? 1 : 0;
    const int narrow = __syncthreads_and(my_narrow);
    T lse_m = T(-INFINITY), lse_s = T(0);
#define YY_PREP_ROWS(M, F, W) \
    prep_rows<T, M, F, W>(k, b, prior_mean, prior_var, bid, nblk, s_hi, s_lo, s_iv, s_cc, s_sc, lse_m, lse_s)
    if (mode == kPrepRestart) {
        if (first) YY_PREP_ROWS(kPrepRestart, true, false);
        else if (narrow) YY_PREP_ROWS(kPrepRestart, false, true);
        else YY_PREP_ROWS(kPrepRestart, false, false);
    } else if (mode == kPrepInit) {
        if (first) YY_PREP_ROWS(kPrepInit, true, false); else YY_PREP_ROWS(kPrepInit, false, false);
    } else {
        if (first) YY_PREP_ROWS(kPrepOnly, true, false);
        else if (narrow) YY_PREP_ROWS(kPrepOnly, false, true);
        else YY_PREP_ROWS(kPrepOnly, false, false);
    }
#undef YY_PREP_ROWS
    if (lse_out && mode != kPrepOnly) {
        __shared__ double sm_m[8], sm_s[8];
        const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
        if (lane == 0) { sm_m[wib] = (double)lse_m; sm_s[wib] = (double)lse_s; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double M = -INFINITY, S = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                const double m2 = sm_m[w], s2 = sm_s[w];
                if (m2 == -INFINITY) continue;
                if (M == -INFINITY) { M = m2; S = s2; }
                else if (m2 > M) { S = S * exp(M - m2) + s2; M = m2; }
                else S += s2 * exp(m2 - M);
            }
            b.part[2 * bid] = M;
            b.part[2 * bid + 1] = S;
        }
    }
}

template <typename T>
__global__ void k_prep_dims(Consts<T> k, Bufs<T> b, int mode, int init_kind) {
    prep_dims_body<T>(k, b, mode, init_kind, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) k_prep(Consts<T> k, Bufs<T> b, int mode, int first, double prior_mean,
                                              double prior_var) {
    prep_body<T>(k, b, mode, first, prior_mean, prior_var, blockIdx.x, gridDim.x, true);
}
// batched restart preparation: trajectory = blockIdx.y
template <typename T>
__global__ void kb_prep_dims(const Traj<T>* __restrict__ tr) {
    const Traj<T>& t = tr[blockIdx.y];
    prep_dims_body<T>(t.k, t.b, kPrepRestart, t.restart_init, 0, 1);
}
template <typename T>
__global__ void __launch_bounds__(256) kb_prep(const Traj<T>* __restrict__ tr) {
    const Traj<T>& t = tr[blockIdx.y];
    prep_body<T>(t.k, t.b, kPrepRestart, 0, 0.0, 1.0, blockIdx.x, gridDim.x, false);
}

template <typename T>
cudaError_t launch_prep_restart_batch(const Traj<T>* d_traj, int B, long long n_pad_max, cudaStream_t s) {
    kb_prep_dims<T><<<dim3(1, B), 256, 0, s>>>(d_traj);
    long long blocks = (n_pad_max * 32 + 255) / 256;
    if (blocks > 64) blocks = 64;
    kb_prep<T><<<dim3((unsigned)blocks, B), 256, 0, s>>>(d_traj);
    return cudaGetLastError();
}
template cudaError_t launch_prep_restart_batch<float>(const Traj<float>*, int, long long, cudaStream_t);
template cudaError_t launch_prep_restart_batch<double>(const Traj<double>*, int, long long, cudaStream_t);

// Blocks of the single-filter preparation pass (one warp per row, at most 8 per SM); also
// the number of log-sum-exp partials it writes.
// One resident wave of the float pass (3 blocks of 256 per SM at its register budget), so
// that no SM runs a partial last wave.
int prep_grid(long long n_pad) {
    long long blocks = (n_pad * 32 + 255) / 256;
    if (blocks > 152 * 3) blocks = 152 * 3;
    return (int)blocks;
}

template <typename T>
cudaError_t launch_prep_mode(const Consts<T>& k, const Bufs<T>& b, int mode, bool first,
                             double prior_mean, double prior_var, int init_kind, cudaStream_t s) {
    // float64 cosine and sine per dimension: one 32-thread block per 32 dimensions
    k_prep_dims<T><<<(unsigned)((k.r_pad + 31) / 32), 32, 0, s>>>(k, b, mode, init_kind);
    k_prep<T><<<(unsigned)prep_grid(k.n_pad), 256, 0, s>>>(k, b, mode, first ? 1 : 0, prior_mean, prior_var);
    return cudaGetLastError();
}

// The rows only (the per-dimension constants already written, as by the restart head).
template <typename T>
cudaError_t launch_prep_rows(const Consts<T>& k, const Bufs<T>& b, int mode, cudaStream_t s) {
    k_prep<T><<<(unsigned)prep_grid(k.n_pad), 256, 0, s>>>(k, b, mode, 0, 0.0, 1.0);
    return cudaGetLastError();
}
template cudaError_t launch_prep_rows<float>(const Consts<float>&, const Bufs<float>&, int, cudaStream_t);

template <typename T>
cudaError_t launch_prep(const Consts<T>& k, const Bufs<T>& b, bool init_weights, bool first,
                        double prior_mean, double prior_var, cudaStream_t s) {
    return launch_prep_mode<T>(k, b, init_weights ? kPrepInit : kPrepOnly, first, prior_mean,
                               prior_var, 0, s);
}
template cudaError_t launch_prep<float>(const Consts<float>&, const Bufs<float>&, bool, bool,
                                        double, double, cudaStream_t);
template cudaError_t launch_prep<double>(const Consts<double>&, const Bufs<double>&, bool, bool,
                                         double, double, cudaStream_t);

template cudaError_t launch_prep_mode<float>(const Consts<float>&, const Bufs<float>&, int, bool,
                                             double, double, int, cudaStream_t);
template cudaError_t launch_prep_mode<double>(const Consts<double>&, const Bufs<double>&, int,
                                              bool, double, double, int, cudaStream_t);

}  // namespace yy
