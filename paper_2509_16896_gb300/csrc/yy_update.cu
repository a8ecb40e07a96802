// Correction, normalisation, estimate and restart test: the online stage and step 4 of
// "Procedure for the Improved Yau-Yau Algorithm", the observation update and normalisation
// of "Log-Domain Computation", and "Local Resampling-Restart Mechanism".
//
// The Ito-corrected log-likelihood h(x).dy - dt/2 |h(x)|^2 is split as
//     lambda(c) + sum_d dh_d (g_d - dt/2 dh_d),   dh_d = h(c_d + u_d) - h(c_d),
//     g_d = dy_d - dt h(c_d),
// which is an exact rewrite: lambda(c) (float64, once per step) absorbs the large common
// part, and the per-node sum has no cancellation (cubic: dh = u (3c^2 + 3cu + u^2); the
// large-scale model's (x - 100)^3 is the same expansion about c - 100).
// The log-weights kept in T are therefore relative to c_ref + lambda(c); the absolute
// normaliser Lambda_k = c_ref + lambda(c) + LSE(relative) is accumulated in float64.
//
// Passes (all coalesced, one warp per node row or one thread per coordinate):
//   obs_prep        g, centre in T, lambda(c)                             (1 block)
//   loglik          ell' = ell_pred + sum_d ..., per-block (max, sum)     (HBM pass over u)
//   lse_merge       Lambda_rel                                            (1 block, float64)
//   moments         ell_hat = ell' - Lambda_rel, w = e^ell_hat; per block the weight sum,
//                   sum of squares, weighted mean and centred second moment of u over
//                   32-row chunks merged with Chan's update                (HBM pass over u)
//   finalize_*      merge of the block moments (Chan, float64): x_hat = c + mean,
//                   v_hat, ESS = W^2 / sum w^2, Z += Lambda, restart test
//
// Every pass is a __device__ body taking the block index and block count explicitly;
// a single-filter __global__ wrapper runs it over blockIdx.x, and a batched wrapper
// (prefix kb_) runs it for trajectory blockIdx.y of a Traj array, so that one launch
// covers a whole batch of ragged filters.
#include "yy_internal.cuh"
#include "yy_prep_dims.cuh"

namespace yy {

template <typename T>
__device__ __forceinline__ T warp_sum_u(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T> __device__ __forceinline__ T sin_u(T x);
template <> __device__ __forceinline__ float sin_u<float>(float x) { return sinf(x); }
template <> __device__ __forceinline__ double sin_u<double>(double x) { return sin(x); }

template <typename T>
__device__ __forceinline__ T exp_t(T x);
template <>
__device__ __forceinline__ float exp_t<float>(float x) { return expf(x); }
template <>
__device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

// merge (m, s) pairs of a log-sum-exp: value = m + log s
__device__ __forceinline__ void lse_merge(double& m, double& s, double m2, double s2) {
    if (m2 == -INFINITY) return;
    if (m == -INFINITY) { m = m2; s = s2; return; }
    if (m2 > m) { s = s * exp(m - m2) + s2; m = m2; }
    else { s += s2 * exp(m2 - m); }
}

// Moment partials: 4 + 2 r_pad doubles per block (the log-sum-exp partials reuse the
// first 2 x (blocks of their pass, at most 4 kNumPartBlocks) doubles earlier in the step).
size_t part_bytes(int r_pad) {
    return (size_t)kNumPartBlocks * (size_t)(4 + 2 * r_pad) * sizeof(double);
}

// ---------------------------------------------------------------------------------------
// bodies
// ---------------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ void obs_prep_body(const Consts<T>& k, const Bufs<T>& b, const double* __restrict__ dy) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int d = threadIdx.x; d < k.r_pad; d += blockDim.x) {
        if (d < k.r) {
            const double c = b.centre[d];
            // h(c) and the centre of the cubic expansion: x^3 about c, (x - 100)^3 about c - 100
            const double cc = (k.model == YY_MODEL_PAPER_E1) ? c - 100.0 : c;
            const double hc = (k.model == YY_MODEL_LINEAR) ? c : cc * cc * cc;
            const double y = dy[d];
            b.dy_last[d] = y;
            b.obs_g[d] = (T)(y - (double)k.dt * hc);
            b.obs_c[d] = (T)cc;
            const double lcd = hc * y - 0.5 * (double)k.dt * hc * hc;
            if (k.noise == YY_NOISE_DIAG) {
                // weighted by 1 / b_d(c); the nodes' own 1 / b_d(x) enters in the likelihood pass
                const double sc = sin(c);
                const double V = (double)k.nz_v * (1.0 + (double)k.nz_vk * sc * sc);
                const double ibc = 1.0 / (V * V);
                b.obs_l[d] = (T)lcd;
                b.obs_ibc[d] = (T)ibc;
                acc += lcd * ibc;
            } else {
                acc += lcd;
            }
        } else {
            b.obs_g[d] = T(0);
            b.obs_c[d] = T(0);
            b.obs_l[d] = T(0);
            b.obs_ibc[d] = T(0);
        }
    }
    acc = warp_sum_u(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum_u(v);
        if (threadIdx.x == 0) b.stats->lam_c = v;
    }
}

// ell'(i) = ell_pred(i) + sum_d dh_d (g_d - dt/2 dh_d); per-block (max, sum) partials.
// One warp per row; lane l holds float2 l + 32 q of the row (the whole row is loaded
// before any arithmetic, so that up to r_pad / 64 loads per lane are in flight); the
// per-step vectors g and c sit in shared memory.  Coordinates r..r_pad-1 are zero in u and
// in g, so they add nothing.
constexpr int kRowQ = YY_MAX_DIM / 64;

// NOISE (diagonal noise coefficients): per coordinate the update is
//     (h_d dy_d - dt/2 h_d^2) / b_d(x) = (l_d + dh_d (g_d - dt/2 dh_d)) / b_d(x),
// l_d = h(c_d) dy_d - dt/2 h(c_d)^2, stored relative to l_d / b_d(c) (whose sum is lambda(c)).
template <typename T, bool NOISE = false>
__device__ __forceinline__ void loglik_body(const Consts<T>& k, const Bufs<T>& b, int bid, int nblk) {
    __shared__ double sm[8], ss[8];
    __shared__ T s_g[YY_MAX_DIM], s_c[YY_MAX_DIM];
    __shared__ T s_l[NOISE ? YY_MAX_DIM : 1], s_ibc[NOISE ? YY_MAX_DIM : 1];
    for (int d = threadIdx.x; d < k.r_pad; d += blockDim.x) {
        s_g[d] = b.obs_g[d];
        s_c[d] = b.obs_c[d];
        if constexpr (NOISE) { s_l[d] = b.obs_l[d]; s_ibc[d] = b.obs_ibc[d]; }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long warp = (bid * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)nblk * blockDim.x) >> 5;
    const T half_dt = T(0.5) * k.dt;
    const bool cubic = k.model != YY_MODEL_LINEAR;   // cubic in u about obs_c
    const int nq = k.r_pad >> 6;
    T m = T(-INFINITY), s = T(0);   // working precision (see below)
    for (long long i = k.row0 + warp; i < k.row1; i += nwarps) {
        const T p = b.logw_pred[i];
        const float2* ui = reinterpret_cast<const float2*>(b.u + (size_t)i * k.r_pad);
        float2 uu[kRowQ];
#pragma unroll
        for (int q = 0; q < kRowQ; ++q) uu[q] = (q < nq) ? ui[lane + 32 * q] : make_float2(0.f, 0.f);
        T acc[2] = {T(0), T(0)};
#pragma unroll
        for (int q = 0; q < kRowQ; ++q) {
            if (q >= nq) break;   // uniform over the warp
            const int d = 64 * q + 2 * lane;
            const T u0 = (T)uu[q].x, u1 = (T)uu[q].y;
            const T c0 = s_c[d], c1 = s_c[d + 1];
            const T h0 = cubic ? u0 * (T(3) * c0 * c0 + T(3) * c0 * u0 + u0 * u0) : u0;
            const T h1 = cubic ? u1 * (T(3) * c1 * c1 + T(3) * c1 * u1 + u1 * u1) : u1;
            if constexpr (NOISE) {
                // 1 / b_d at the node x = c + u (padded coordinates: u = l = 0, no term)
                const T sx0 = sin_u<T>(c0 + u0), sx1 = sin_u<T>(c1 + u1);
                const T v0 = k.nz_v * (T(1) + k.nz_vk * sx0 * sx0), v1 = k.nz_v * (T(1) + k.nz_vk * sx1 * sx1);
                const T ib0 = T(1) / (v0 * v0), ib1 = T(1) / (v1 * v1);
                acc[q & 1] += (s_l[d] + h0 * (s_g[d] - half_dt * h0)) * ib0 - s_l[d] * s_ibc[d] +
                              (s_l[d + 1] + h1 * (s_g[d + 1] - half_dt * h1)) * ib1 - s_l[d + 1] * s_ibc[d + 1];
            } else {
                acc[q & 1] += h0 * (s_g[d] - half_dt * h0) + h1 * (s_g[d + 1] - half_dt * h1);
            }
        }
        T tot = acc[0] + acc[1];
        tot = warp_sum_u(tot);
        const T lw = (p == T(-INFINITY)) ? T(-INFINITY) : p + tot;
        if (lane == 0) {
            b.logw[i] = lw;
            // running (max, sum) of this warp's rows in the working precision (float64 issue
            // time per row is large on this part); blocks merge in float64
            if (lw != T(-INFINITY)) {
                if (lw > m) {
                    s = (m == T(-INFINITY)) ? T(1) : s * exp_t<T>(m - lw) + T(1);
                    m = lw;
                } else {
                    s += exp_t<T>(lw - m);
                }
            }
        }
    }
    if (lane == 0) { sm[wib] = (double)m; ss[wib] = (double)s; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double M = -INFINITY, S = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) lse_merge(M, S, sm[w], ss[w]);
        b.part[2 * bid] = M;
        b.part[2 * bid + 1] = S;
    }
}

// LSE partials of b.logw (used after init / restart weights).
template <typename T>
__device__ __forceinline__ void lse_partials_body(const Consts<T>& k, const Bufs<T>& b, int conditional, int bid,
                                                  int nblk) {
    if (conditional && b.stats->restart_flag == 0) return;
    __shared__ double sm[8], ss[8];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double m = -INFINITY, s = 0.0;
    for (long long i = bid * (long long)blockDim.x + threadIdx.x; i < k.n; i += (long long)nblk * blockDim.x)
        lse_merge(m, s, (double)b.logw[i], 1.0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double m2 = __shfl_xor_sync(0xffffffffu, m, o);
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
        lse_merge(m, s, m2, s2);
    }
    if (lane == 0) { sm[wib] = m; ss[wib] = s; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double M = -INFINITY, S = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) lse_merge(M, S, sm[w], ss[w]);
        b.part[2 * bid] = M;
        b.part[2 * bid + 1] = S;
    }
}

// The partials' maxima and sums are float64; the rescale factors e^(m_b - M) in [0, 1]
// are taken in the filter's working precision T (a float64 exponential per partial is
// costly on this part, and float filters carry their log-weights in float).
template <typename T>
__device__ __forceinline__ void lse_merge_body(const double* __restrict__ part, int nb, DevStats* st, int conditional,
                                               int report = 1) {
    if (conditional && st->restart_flag == 0) return;
    __shared__ double red[32];
    __shared__ double s_max;
    // phase 1: the largest block maximum
    double m = -INFINITY;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) m = fmax(m, part[2 * i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double M = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) M = fmax(M, red[w]);
        s_max = M;
    }
    __syncthreads();
    const double M = s_max;
    // phase 2: sum of the block sums rescaled to M
    double s = 0.0;
    if (M != -INFINITY)
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            const double mb = part[2 * i];
            if (mb != -INFINITY)
                s += part[2 * i + 1] * (sizeof(T) == 4 ? (double)expf((float)(mb - M)) : exp(mb - M));
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) S += red[w];
        if (M == -INFINITY) {
            if (report) st->status |= kStatusDegenerate;   // a shard's own rows may all be empty
            st->lam_rel = 0.0;
        } else {
            st->lam_rel = M + log(S);
            if (!isfinite(st->lam_rel)) { st->status |= kStatusNonFinite; st->lam_rel = 0.0; }
        }
    }
}

template <typename T>
__device__ __forceinline__ void subtract_body(const Consts<T>& k, const Bufs<T>& b, int conditional, int bid,
                                              int nblk) {
    if (conditional && b.stats->restart_flag == 0) return;
    const T lam = (T)b.stats->lam_rel;
    for (long long i = bid * (long long)blockDim.x + threadIdx.x; i < k.n; i += (long long)nblk * blockDim.x)
        b.logw[i] = b.logw[i] - lam;
}

constexpr int kMomDims = YY_MAX_DIM / 256;   // coordinates per thread in the moments pass

// Normalises ell' and accumulates per-block weighted moments of u.  The block's rows are
// taken 256 at a time (one per thread): ell_hat = ell' - Lambda_rel and w = e^ell_hat, the
// round's weight sum and sum of squares (float64), and the rows with w > 0 compacted in
// row order (ballot prefix sums, so the result does not depend on scheduling).  Only those
// rows are read: per coordinate the round's weighted mean, then its centred second moment,
// merged into the block's running values with Chan's rule (float64).  With posteriors
// concentrated on few nodes most rounds read no coordinates at all.
template <typename T>
__device__ __forceinline__ void moments_body(const Consts<T>& k, const Bufs<T>& b, int bid, int nblk) {
    __shared__ int s_rows[256];
    __shared__ T s_w[256];
    __shared__ int s_wcnt[8];
    __shared__ double s_red[2][8];
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const long long rows_per = (k.row1 - k.row0 + nblk - 1) / nblk;
    const long long i0 = k.row0 + bid * rows_per;
    const long long i1 = min(k.row1, i0 + rows_per);
    const T lam = (T)b.stats->lam_rel;
    double W = 0.0, Q = 0.0;
    double mu[kMomDims], M2[kMomDims];
#pragma unroll
    for (int q = 0; q < kMomDims; ++q) { mu[q] = 0.0; M2[q] = 0.0; }
    for (long long c0 = i0; c0 < i1; c0 += 256) {
        const long long i = c0 + tid;
        T w = T(0);
        if (i < i1) {
            const T lh = b.logw[i] - lam;
            b.logw[i] = lh;
            w = exp_t<T>(lh);
        }
        // round sums and the compacted list of rows with weight
        const double wsum = warp_sum_u((double)w), wsq = warp_sum_u((double)w * (double)w);
        const uint32_t bal = __ballot_sync(0xffffffffu, w > T(0));
        if (lane == 0) { s_red[0][wib] = wsum; s_red[1][wib] = wsq; s_wcnt[wib] = __popc(bal); }
        __syncthreads();
        int off = 0, cnt = 0;
        double Wc = 0.0, Qc = 0.0;
        for (int g = 0; g < 8; ++g) {
            if (g < wib) off += s_wcnt[g];
            cnt += s_wcnt[g];
            Wc += s_red[0][g];
            Qc += s_red[1][g];
        }
        if (w > T(0)) {
            const int slot = off + __popc(bal & ((1u << lane) - 1u));
            s_rows[slot] = (int)(i - c0);
            s_w[slot] = w;
        }
        __syncthreads();
        if (cnt > 0 && Wc > 0.0) {
            // every coordinate slot of this thread in one sweep over the rows (its loads in
            // flight together); per slot the sums run over the rows in the same order
            T S[kMomDims], muc[kMomDims], m2[kMomDims];
#pragma unroll
            for (int q = 0; q < kMomDims; ++q) { S[q] = T(0); m2[q] = T(0); }
#pragma unroll 4   // several rows' loads in flight; the sums still run in row order
            for (int l = 0; l < cnt; ++l) {
                const float* ur = b.u + (size_t)(c0 + s_rows[l]) * k.r_pad;
                const T wl = s_w[l];
#pragma unroll
                for (int q = 0; q < kMomDims; ++q) {
                    const int d = tid + 256 * q;
                    if (d < k.r) S[q] += wl * (T)ur[d];
                }
            }
#pragma unroll
            for (int q = 0; q < kMomDims; ++q) muc[q] = S[q] / (T)Wc;
#pragma unroll 4
            for (int l = 0; l < cnt; ++l) {
                const float* ur = b.u + (size_t)(c0 + s_rows[l]) * k.r_pad;
                const T wl = s_w[l];
#pragma unroll
                for (int q = 0; q < kMomDims; ++q) {
                    const int d = tid + 256 * q;
                    if (d < k.r) {
                        const T dv = (T)ur[d] - muc[q];
                        m2[q] += wl * dv * dv;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kMomDims; ++q) {
                const int d = tid + 256 * q;
                if (d < k.r) {
                    const double delta = (double)muc[q] - mu[q];
                    const double Wn = W + Wc;
                    mu[q] += delta * (Wc / Wn);
                    M2[q] += (double)m2[q] + delta * delta * (W * Wc / Wn);
                }
            }
            W += Wc;
        }
        Q += Qc;
        __syncthreads();
    }
    double* p = b.part + (size_t)bid * (4 + 2 * k.r_pad);
    if (tid == 0) { p[0] = W; p[1] = Q; }
    // only partials with weight are merged (finalize_scalars lists them), so a block
    // without weight -- most of them when the posterior is concentrated -- writes no moments
    if (W > 0.0) {
#pragma unroll
        for (int q = 0; q < kMomDims; ++q) {
            const int d = tid + 256 * q;
            if (d < k.r_pad) { p[4 + d] = mu[q]; p[4 + k.r_pad + d] = M2[q]; }
        }
    }
}

// Scalars of the step: weight sum W and sum of squares Q over the block partials,
// ESS = W^2 / Q, Lambda = c_ref + lambda(c) + Lambda_rel, Z += Lambda, step k += 1 and the
// restart test.
// rec != NULL (a shard of a row-split filter): the head of the shard's record (its
// log-sum-exp, W, Q) is written instead of the step's scalars, which the merge of all
// shards' records sets.
template <typename T>
__device__ __forceinline__ void finalize_scalars_body(const Consts<T>& k, const Bufs<T>& b, int nb,
                                                      int restart_interval, double ess_frac, double* rec = nullptr) {
    __shared__ double red_w[32], red_q[32];
    __shared__ int s_cnt[32];
    DevStats* st = b.stats;
    const int t = threadIdx.x;
    double w = 0.0, q = 0.0;
    // partials with weight, listed in block order for the per-coordinate merge (nb <= blockDim.x)
    bool has = false;
    if (t < nb) {
        const double* p = b.part + (size_t)t * (4 + 2 * k.r_pad);
        has = p[0] > 0.0;
        if (has) w += p[0];
        q += p[1];
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, has);
    if ((t & 31) == 0) s_cnt[t >> 5] = __popc(bal);
    __syncthreads();
    {
        int off = 0, tot = 0;
        for (int g = 0; g < (int)(blockDim.x >> 5); ++g) {
            if (g < (t >> 5)) off += s_cnt[g];
            tot += s_cnt[g];
        }
        if (has) b.part_list[off + __popc(bal & ((1u << (t & 31)) - 1u))] = t;
        if (t == 0) st->part_count = tot;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        w += __shfl_xor_sync(0xffffffffu, w, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
    }
    if ((t & 31) == 0) { red_w[t >> 5] = w; red_q[t >> 5] = q; }
    __syncthreads();
    if (t == 0 && rec) {
        double W = 0.0, Q = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { W += red_w[i]; Q += red_q[i]; }
        rec[0] = st->lam_rel;
        rec[1] = W;
        rec[2] = Q;
        rec[3] = 0.0;
    } else if (t == 0) {
        double W = 0.0, Q = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { W += red_w[i]; Q += red_q[i]; }
        st->wsum = W;
        st->wsq = Q;
        const double ess = (Q > 0.0) ? W * W / Q : 0.0;
        st->ess = ess;
        const double lam = st->c_ref + st->lam_c + st->lam_rel;
        st->lam = lam;
        st->lognorm += lam;
        if (!isfinite(lam)) st->status |= kStatusNonFinite;
        st->step += 1;
        const bool by_ess = ess_frac > 0.0 && ess < ess_frac * (double)k.n;
        const bool by_int = restart_interval >= 2 && (st->step % restart_interval) == 0;
        st->restart_flag = (by_ess || by_int) ? 1 : 0;
    }
}

// Per coordinate: mean and variance from the block partials with weight (finalize_scalars'
// list), one warp per coordinate, 8 per block, in two reductions: the mean of the block
// means weighted by W_b (one division), then M2 = sum of M2_b + W_b (mu_b - mu)^2 about it
// (the parallel-axis identity: the same quantity as merging the partials pairwise, without a
// float64 division per partial, slow on this part); x_hat = c + mean.
// rec != NULL: the shard's merged mean and M2 of u go to its record instead of x_hat, v_hat.
template <typename T>
__device__ __forceinline__ void finalize_dims_body(const Consts<T>& k, const Bufs<T>& b, int nb, int bid,
                                                   double* rec = nullptr) {
    (void)nb;
    const int lane = threadIdx.x & 31;
    const int d = bid * 8 + (int)(threadIdx.x >> 5);
    if (d >= k.r) return;
    const int np = b.stats->part_count;
    const size_t stride = 4 + 2 * (size_t)k.r_pad;
    double W = 0.0, WM = 0.0;
    for (int jj = lane; jj < np; jj += 32) {
        const double* p = b.part + (size_t)b.part_list[jj] * stride;
        W += p[0];
        WM = fma(p[0], p[4 + d], WM);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        W += __shfl_xor_sync(0xffffffffu, W, o);
        WM += __shfl_xor_sync(0xffffffffu, WM, o);
    }
    const double mu = (W > 0.0) ? WM / W : 0.0;
    double M2 = 0.0;
    for (int jj = lane; jj < np; jj += 32) {
        const double* p = b.part + (size_t)b.part_list[jj] * stride;
        const double dm = p[4 + d] - mu;
        M2 += fma(p[0] * dm, dm, p[4 + k.r_pad + d]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) M2 += __shfl_xor_sync(0xffffffffu, M2, o);
    if (lane != 0) return;
    if (rec) {
        rec[4 + d] = mu;
        rec[4 + k.r + d] = M2;
    } else {
        const double mean = b.centre[d] + mu;
        const double var = (W > 0.0) ? M2 / W : 0.0;
        b.mean[d] = mean;
        b.var[d] = var;
        if (!isfinite(mean) || !isfinite(var)) atomicOr(&b.stats->status, kStatusNonFinite);
    }
}

__device__ __forceinline__ void restart_begin_body(DevStats* st, int mode) {
    if (threadIdx.x != 0) return;
    if (mode == YY_RESTART_FORCE) st->restart_flag = 1;
    st->last_restarted = 0;
}

// Box of the restart in progress.  Plain rule: centre x_hat, half-widths unchanged.
// Learned rule (out = network output [delta; lambda], or NULL): centre x_hat + delta,
// half-widths base_R exp(lambda), accepted only if every value is finite, every
// half-width lies in [base_R / 8, 8 base_R] and the box contains x_hat (|delta_d| <= half-
// width); the offset c_ref follows the box volume.
template <typename T>
__device__ __forceinline__ void restart_box_body(const Consts<T>& k, const Bufs<T>& b, const float* out,
                                                 double base_R) {
    __shared__ int s_ok;
    if (b.stats->restart_flag == 0) return;
    if (threadIdx.x == 0) s_ok = (out != nullptr) ? 1 : 0;
    __syncthreads();
    if (out) {
        for (int d = threadIdx.x; d < k.r; d += blockDim.x) {
            const double delta = (double)out[d], lam = (double)out[k.r + d];
            const double h = base_R * exp(lam);
            if (!isfinite(delta) || !isfinite(h) || h < base_R / 8.0 || h > 8.0 * base_R || fabs(delta) > h)
                atomicAnd(&s_ok, 0);
        }
        __syncthreads();
    }
    const bool learned = s_ok != 0;
    __shared__ double red[32];
    double dl = 0.0;
    int changed = 0;
    for (int d = threadIdx.x; d < k.r_pad; d += blockDim.x) {
        double c = 0.0, h = b.halfwidth[d];
        if (d < k.r) {
            c = b.mean[d];
            if (learned) {
                c += (double)out[d];
                h = base_R * exp((double)out[k.r + d]);
                dl += log(h / b.halfwidth[d]);
                changed |= (h != b.halfwidth[d]);
            }
        }
        b.next_centre[d] = c;
        b.next_half[d] = h;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dl += __shfl_xor_sync(0xffffffffu, dl, o);
    changed = __any_sync(0xffffffffu, changed);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dl;
    __shared__ int s_changed;
    if (threadIdx.x == 0) s_changed = 0;
    __syncthreads();
    if (changed && (threadIdx.x & 31) == 0) atomicOr(&s_changed, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        b.stats->c_ref += tot;
        b.stats->scale_changed = s_changed;
    }
}

template <typename T>
__device__ __forceinline__ void restart_commit_body(const Consts<T>& k, const Bufs<T>& b) {
    if (b.stats->restart_flag == 0) return;
    for (int d = threadIdx.x; d < k.r_pad; d += blockDim.x) {
        b.centre[d] = b.next_centre[d];
        b.halfwidth[d] = b.next_half[d];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        b.stats->restarts += 1;
        b.stats->restart_flag = 0;
        b.stats->last_restarted = 1;
        b.stats->op_stale = 1;   // the nodes moved: a materialised operator is rebuilt
    }
}

// Row of the estimate history: x_hat[r], v_hat[r], ESS, Lambda, Z, restart test result.
template <typename T>
__device__ __forceinline__ void record_body(const Consts<T>& k, const Bufs<T>& b, double* __restrict__ row) {
    for (int d = threadIdx.x; d < k.r; d += blockDim.x) {
        row[d] = b.mean[d];
        row[k.r + d] = b.var[d];
    }
    if (threadIdx.x == 0) {
        row[2 * k.r] = b.stats->ess;
        row[2 * k.r + 1] = b.stats->lam;
        row[2 * k.r + 2] = b.stats->lognorm;
        row[2 * k.r + 3] = b.stats->restart_flag ? 1.0 : 0.0;
    }
}

// ---------------------------------------------------------------------------------------
// single-filter wrappers
// ---------------------------------------------------------------------------------------

template <typename T>
__global__ void k_obs_prep(Consts<T> k, Bufs<T> b, const double* __restrict__ dy) { obs_prep_body<T>(k, b, dy); }
template <typename T, bool NOISE = false>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_loglik(Consts<T> k, Bufs<T> b) {
    loglik_body<T, NOISE>(k, b, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(256) k_lse_partials(Consts<T> k, Bufs<T> b, int conditional) {
    lse_partials_body<T>(k, b, conditional, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void k_lse_merge(const double* __restrict__ part, int nb, DevStats* st, int conditional, int report = 1) {
    lse_merge_body<T>(part, nb, st, conditional, report);
}
template <typename T>
__global__ void k_subtract(Consts<T> k, Bufs<T> b, int conditional) {
    subtract_body<T>(k, b, conditional, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(256) k_moments(Consts<T> k, Bufs<T> b) { moments_body<T>(k, b, blockIdx.x, gridDim.x); }
template <typename T>
__global__ void __launch_bounds__(512) k_finalize_scalars(Consts<T> k, Bufs<T> b, int nb, int restart_interval,
                                                          double ess_frac, double* rec = nullptr) {
    finalize_scalars_body<T>(k, b, nb, restart_interval, ess_frac, rec);
}
template <typename T>
__global__ void __launch_bounds__(256) k_finalize_dims(Consts<T> k, Bufs<T> b, int nb, double* rec = nullptr) {
    finalize_dims_body<T>(k, b, nb, blockIdx.x, rec);
}
template <typename T>
__global__ void k_restart_begin(DevStats* st, int mode) { restart_begin_body(st, mode); }
// Float filters without a learned proposal: the restart decision, the box at x_hat and the
// restart pass's per-dimension constants in one block (the three steps of k_restart_begin,
// k_restart_box and k_prep_dims; each reads what the one before wrote).
template <typename T>
__global__ void __launch_bounds__(256) k_restart_head(Consts<T> k, Bufs<T> b, int mode, int init_kind,
                                                      double base_R) {
    restart_begin_body(b.stats, mode);
    __syncthreads();
    restart_box_body<T>(k, b, nullptr, base_R);
    __syncthreads();
    prep_dims_body<T>(k, b, kPrepRestart, init_kind, 0, 1);
}
template <typename T>
__global__ void k_restart_commit(Consts<T> k, Bufs<T> b) { restart_commit_body<T>(k, b); }
template <typename T>
__global__ void k_restart_box(Consts<T> k, Bufs<T> b, const float* out, double base_R) {
    restart_box_body<T>(k, b, out, base_R);
}
template <typename T>
__global__ void k_record(Consts<T> k, Bufs<T> b, double* __restrict__ row) { record_body<T>(k, b, row); }

// ---------------------------------------------------------------------------------------
// batched wrappers: trajectory = blockIdx.y
// ---------------------------------------------------------------------------------------

template <typename T>
__global__ void kb_obs_prep(const Traj<T>* __restrict__ tr, const double* __restrict__ dy_row) {
    const Traj<T>& t = tr[blockIdx.y];
    obs_prep_body<T>(t.k, t.b, dy_row + t.dy_off);
}
template <typename T>
__global__ void __launch_bounds__(256) kb_loglik(const Traj<T>* __restrict__ tr) {
    const Traj<T>& t = tr[blockIdx.y];
    loglik_body<T>(t.k, t.b, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void kb_lse_merge(const Traj<T>* __restrict__ tr, int nb, int conditional) {
    const Traj<T>& t = tr[blockIdx.y];
    lse_merge_body<T>(t.b.part, nb, t.b.stats, conditional);
}
template <typename T>
__global__ void __launch_bounds__(256) kb_moments(const Traj<T>* __restrict__ tr) {
    const Traj<T>& t = tr[blockIdx.y];
    moments_body<T>(t.k, t.b, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void __launch_bounds__(512) kb_finalize_scalars(const Traj<T>* __restrict__ tr, int nb) {
    const Traj<T>& t = tr[blockIdx.y];
    finalize_scalars_body<T>(t.k, t.b, nb, t.restart_interval, t.ess_frac);
}
template <typename T>
__global__ void __launch_bounds__(256) kb_finalize_dims(const Traj<T>* __restrict__ tr, int nb) {
    const Traj<T>& t = tr[blockIdx.y];
    finalize_dims_body<T>(t.k, t.b, nb, blockIdx.x);
}
template <typename T>
__global__ void kb_record(const Traj<T>* __restrict__ tr, double* __restrict__ hist_row) {
    const Traj<T>& t = tr[blockIdx.y];
    record_body<T>(t.k, t.b, hist_row + t.hist_off);
}
template <typename T>
__global__ void kb_reset(const Traj<T>* __restrict__ tr, int B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    tr[i].b.stats->clamps = 0u;
    tr[i].b.stats->candidates = 0ull;
}
template <typename T>
__global__ void kb_restart_begin(const Traj<T>* __restrict__ tr) { restart_begin_body(tr[blockIdx.y].b.stats, YY_RESTART_AUTO); }
template <typename T>
__global__ void __launch_bounds__(256) kb_lse_partials(const Traj<T>* __restrict__ tr) {
    const Traj<T>& t = tr[blockIdx.y];
    lse_partials_body<T>(t.k, t.b, 1, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void kb_subtract(const Traj<T>* __restrict__ tr) {
    const Traj<T>& t = tr[blockIdx.y];
    subtract_body<T>(t.k, t.b, 1, blockIdx.x, gridDim.x);
}
template <typename T>
__global__ void kb_restart_box(const Traj<T>* __restrict__ tr) {
    const Traj<T>& t = tr[blockIdx.y];
    restart_box_body<T>(t.k, t.b, nullptr, 0.0);
}
template <typename T>
__global__ void kb_restart_commit(const Traj<T>* __restrict__ tr) {
    const Traj<T>& t = tr[blockIdx.y];
    restart_commit_body<T>(t.k, t.b);
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------

template <typename T>
cudaError_t launch_update(const Consts<T>& k, const Bufs<T>& b, const double* dy,
                          int restart_interval, double ess_frac, cudaStream_t s, int* launches) {
    const int nb = kNumPartBlocks;
    // the likelihood pass runs one wave of blocks: 4 per SM in float (64 registers a
    // thread), 2 in double (its partials are 2 doubles per block, well inside the moment
    // partials' space)
    const int nbl = (sizeof(T) == 4 ? 2 : 1) * kNumPartBlocks;
    k_obs_prep<T><<<1, 256, 0, s>>>(k, b, dy);
    if (k.noise == YY_NOISE_DIAG) k_loglik<T, true><<<nbl, 256, 0, s>>>(k, b);
    else k_loglik<T><<<nbl, 256, 0, s>>>(k, b);
    k_lse_merge<T><<<1, 256, 0, s>>>(b.part, nbl, b.stats, 0);
    k_moments<T><<<nb, 256, 0, s>>>(k, b);
    k_finalize_scalars<T><<<1, 512, 0, s>>>(k, b, nb, restart_interval, ess_frac);
    k_finalize_dims<T><<<(k.r + 7) / 8, 256, 0, s>>>(k, b, nb);
    if (launches) *launches += 6;
    return cudaGetLastError();
}

// One shard of a row-split filter: the same passes over the shard's rows (k.row0..k.row1),
// its log-weights normalised by its own log-sum-exp, and its record written to rec
// (2r + 4 doubles, yy_shard.cuh) instead of the step's scalars and estimate.
template <typename T>
cudaError_t launch_update_shard(const Consts<T>& k, const Bufs<T>& b, const double* dy, double* rec, cudaStream_t s,
                                int* launches) {
    const int nb = kNumPartBlocks;
    const int nbl = (sizeof(T) == 4 ? 2 : 1) * kNumPartBlocks;
    k_obs_prep<T><<<1, 256, 0, s>>>(k, b, dy);
    if (k.noise == YY_NOISE_DIAG) k_loglik<T, true><<<nbl, 256, 0, s>>>(k, b);
    else k_loglik<T><<<nbl, 256, 0, s>>>(k, b);
    k_lse_merge<T><<<1, 256, 0, s>>>(b.part, nbl, b.stats, 0, 0);
    k_moments<T><<<nb, 256, 0, s>>>(k, b);
    k_finalize_scalars<T><<<1, 512, 0, s>>>(k, b, nb, 0, 0.0, rec);
    k_finalize_dims<T><<<(k.r + 7) / 8, 256, 0, s>>>(k, b, nb, rec);
    if (launches) *launches += 6;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_normalise_only(const Consts<T>& k, const Bufs<T>& b, cudaStream_t s,
                                  int* launches) {
    const int nb = kNumPartBlocks;
    k_lse_partials<T><<<nb, 256, 0, s>>>(k, b, 0);
    k_lse_merge<T><<<1, 256, 0, s>>>(b.part, nb, b.stats, 0);
    k_subtract<T><<<nb, 256, 0, s>>>(k, b, 0);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_record(const Consts<T>& k, const Bufs<T>& b, double* hist_row, cudaStream_t s) {
    k_record<T><<<1, 256, 0, s>>>(k, b, hist_row);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prep_mode(const Consts<T>& k, const Bufs<T>& b, int mode, bool first,
                             double prior_mean, double prior_var, int init_kind, cudaStream_t s);
template <typename T>
cudaError_t launch_prep_rows(const Consts<T>& k, const Bufs<T>& b, int mode, cudaStream_t s);
template <typename T>
cudaError_t launch_prep_restart_batch(const Traj<T>* d_traj, int B, long long n_pad_max, cudaStream_t s);

// Restart sequence (every kernel is a no-op unless the restart flag is set): begin, the
// learned proposal (network forward pass, if a network is attached), the box, re-mapping of
// the nodes when the half-widths change, preparation at the new box, weights, commit.
template <typename T>
cudaError_t launch_restart(const Consts<T>& k, const Bufs<T>& b, int mode, int init_kind, double base_R,
                           struct ::yy_mlp* net, cudaStream_t s, int* launches) {
    if (mode == YY_RESTART_NEVER) return cudaSuccess;
    const int nb = kNumPartBlocks;
    if (!net && sizeof(T) == 4) {   // float, plain or Gaussian restart: head, rows, weights, commit
        k_restart_head<T><<<1, 256, 0, s>>>(k, b, mode, init_kind, base_R);
        cudaError_t e = launch_prep_rows<T>(k, b, 2 /*restart*/, s);
        if (e != cudaSuccess) return e;
        k_lse_merge<T><<<1, 256, 0, s>>>(b.part, prep_grid(k.n_pad), b.stats, 1);
        k_subtract<T><<<nb, 256, 0, s>>>(k, b, 1);
        k_restart_commit<T><<<1, 256, 0, s>>>(k, b);
        if (launches) *launches += 5;
        return cudaGetLastError();
    }
    int l = 0;
    k_restart_begin<T><<<1, 32, 0, s>>>(b.stats, mode);
    const float* out = nullptr;
    if (net) {
        cudaError_t e = mlp_propose(net, k.r, b.mean, b.var, b.dy_last, b.centre, (double)k.dt, &b.stats->restart_flag, s, &l);
        if (e != cudaSuccess) return e;
        out = mlp_output(net);
    }
    k_restart_box<T><<<1, 256, 0, s>>>(k, b, out, base_R);
    cudaError_t e = cudaSuccess;
    if (net) e = launch_sobol_points_restart(b.dirs, k.r, k.r_pad, k.n, b.u, b.next_half, b.stats, s);
    if (e != cudaSuccess) return e;
    e = launch_prep_mode<T>(k, b, 2 /*restart*/, false, 0.0, 1.0, init_kind, s);
    if (e != cudaSuccess) return e;
    // the preparation pass wrote the log-sum-exp partials of the new weights
    k_lse_merge<T><<<1, 256, 0, s>>>(b.part, prep_grid(k.n_pad), b.stats, 1);
    k_subtract<T><<<nb, 256, 0, s>>>(k, b, 1);
    k_restart_commit<T><<<1, 256, 0, s>>>(k, b);
    if (launches) *launches += 7 + l + (net ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_batch(const Traj<T>* d_traj, int B, int r_max, const double* dy_row,
                                int nbu, cudaStream_t s, int* launches) {
    const dim3 one(1, B), many(nbu, B);
    kb_obs_prep<T><<<one, 256, 0, s>>>(d_traj, dy_row);
    kb_loglik<T><<<many, 256, 0, s>>>(d_traj);
    kb_lse_merge<T><<<one, 256, 0, s>>>(d_traj, nbu, 0);
    kb_moments<T><<<many, 256, 0, s>>>(d_traj);
    kb_finalize_scalars<T><<<one, 512, 0, s>>>(d_traj, nbu);
    kb_finalize_dims<T><<<dim3((r_max + 7) / 8, B), 256, 0, s>>>(d_traj, nbu);
    if (launches) *launches += 6;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restart_batch(const Traj<T>* d_traj, int B, int r_max, long long n_pad_max,
                                 int nbu, cudaStream_t s, int* launches) {
    (void)r_max;
    const dim3 one(1, B), many(nbu, B);
    kb_restart_begin<T><<<one, 32, 0, s>>>(d_traj);
    kb_restart_box<T><<<one, 256, 0, s>>>(d_traj);
    cudaError_t e = launch_prep_restart_batch<T>(d_traj, B, n_pad_max, s);
    if (e != cudaSuccess) return e;
    kb_lse_partials<T><<<many, 256, 0, s>>>(d_traj);
    kb_lse_merge<T><<<one, 256, 0, s>>>(d_traj, nbu, 1);
    kb_subtract<T><<<many, 256, 0, s>>>(d_traj);
    kb_restart_commit<T><<<one, 256, 0, s>>>(d_traj);
    if (launches) *launches += 8;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_record_batch(const Traj<T>* d_traj, int B, double* hist_row, cudaStream_t s, int* launches) {
    kb_record<T><<<dim3(1, B), 256, 0, s>>>(d_traj, hist_row);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reset_batch(const Traj<T>* d_traj, int B, cudaStream_t s, int* launches) {
    kb_reset<T><<<(B + 127) / 128, 128, 0, s>>>(d_traj, B);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

#define YY_INST(T)                                                                                      \
    template cudaError_t launch_record<T>(const Consts<T>&, const Bufs<T>&, double*, cudaStream_t);     \
    template cudaError_t launch_update<T>(const Consts<T>&, const Bufs<T>&, const double*, int, double, \
                                          cudaStream_t, int*);                                          \
    template cudaError_t launch_normalise_only<T>(const Consts<T>&, const Bufs<T>&, cudaStream_t, int*); \
    template cudaError_t launch_update_shard<T>(const Consts<T>&, const Bufs<T>&, const double*, double*,     \
                                                cudaStream_t, int*);                                            \
    template cudaError_t launch_restart<T>(const Consts<T>&, const Bufs<T>&, int, int, double, struct ::yy_mlp*, \
                                           cudaStream_t, int*);                                          \
    template cudaError_t launch_update_batch<T>(const Traj<T>*, int, int, const double*, int, cudaStream_t, \
                                                int*);                                                  \
    template cudaError_t launch_restart_batch<T>(const Traj<T>*, int, int, long long, int, cudaStream_t,  \
                                                 int*);                                                 \
    template cudaError_t launch_record_batch<T>(const Traj<T>*, int, double*, cudaStream_t, int*);      \
    template cudaError_t launch_reset_batch<T>(const Traj<T>*, int, cudaStream_t, int*);
YY_INST(float)
YY_INST(double)
#undef YY_INST

}  // namespace yy
