// Per-dimension constants of the preparation pass, shared by the pass's own launch and the
// restart's head kernel.
#pragma once

#include "yy_internal.cuh"
#include "yy_drift.cuh"

namespace yy {

enum PrepMode { kPrepOnly = 0, kPrepInit = 1, kPrepRestart = 2 };

// cos c and sin c of a centre coordinate, rounded to the working precision.  Float: from
// sincosf of the float head of c with its tail as a first-order correction (the tail is
// below half an ulp of the head, so the neglected terms are under float rounding) -- a
// float64 sine and cosine per coordinate cost more than the whole restart head on this
// part; double: sin, cos.
template <typename T>
__device__ __forceinline__ void dim_cos_sin(double c, T* cs, T* sn);
template <>
__device__ __forceinline__ void dim_cos_sin<float>(double c, float* cs, float* sn) {
    const float hi = (float)c;
    const float lo = (float)(c - (double)hi);
    float s, co;
    sincosf(hi, &s, &co);
    *cs = fmaf(-s, lo, co);
    *sn = fmaf(co, lo, s);
}
template <>
__device__ __forceinline__ void dim_cos_sin<double>(double c, double* cs, double* sn) {
    sincos(c, sn, cs);
}

// Per-dimension constants of one preparation pass: the centre split into a T-precision
// head and tail (x = c_hi + (u + c_lo) loses only the final rounding), for a Gaussian
// restart 1 / (2 max(v_hat_d, (R_d / 4)^2)), and cos c_d, sin c_d (NaN cosine where the
// half-width is too wide for the polynomials of yy_drift.cuh).
template <typename T>
__device__ __forceinline__ void prep_dims_body(const Consts<T>& k, const Bufs<T>& b, int mode, int init_kind,
                                               int bid, int nblk) {
    if (mode == kPrepRestart && b.stats->restart_flag == 0) return;
    const double* cen = (mode == kPrepRestart) ? b.next_centre : b.centre;
    const double* half = (mode == kPrepRestart) ? b.next_half : b.halfwidth;
    const int rp = k.r_pad;
    for (int d = bid * blockDim.x + threadIdx.x; d < rp; d += nblk * blockDim.x) {
        T hi = T(0), lo = T(0), iv = T(0), cc = T(0), sc = T(0);   // padded: u = 0 gives f = 0
        if (d < k.r) {
            const double c = cen[d];
            hi = (T)c;
            lo = (T)(c - (double)hi);
            if (mode == kPrepRestart && init_kind == YY_RESTART_INIT_GAUSS) {
                const double R4 = 0.25 * half[d];
                iv = (T)(0.5 / fmax(b.var[d], R4 * R4));
            }
            T cs, sn;
            dim_cos_sin<T>(c, &cs, &sn);
            cc = (half[d] <= kPolyMaxU) ? cs : (T)NAN;
            sc = sn;
        }
        b.dimc[d] = hi;
        b.dimc[rp + d] = lo;
        b.dimc[2 * rp + d] = iv;
        b.dimc[3 * rp + d] = cc;
        b.dimc[4 * rp + d] = sc;
    }
}

}  // namespace yy
