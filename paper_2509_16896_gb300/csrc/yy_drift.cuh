// Drift of the cubic sensor model ("Large-Scale Scalability Test"), f_d(x) = cos x_d, and
// sin x_d (for the divergence), in float32 at x_d = c_d + u from per-dimension constants of the box:
//     cos(c + u) = cos c cos u - sin c sin u,    sin(c + u) = sin c cos u + cos c sin u,
// with cos c, sin c taken once per dimension in float64 and cos u, sin u from their Taylor
// polynomials through u^8 and u^9 (Horner in u^2).  For |u| <= kPolyMaxU = 0.6 the
// truncation error is below 2e-9, under float32 rounding.  A dimension whose box half-width
// exceeds kPolyMaxU carries cc = NaN and is evaluated by sincosf of x = hi + (u + lo) (the
// centre split into a float head and tail).  The preparation pass and the exact pair
// evaluation of the BF16 screen both call this, so the drift they use is the same value.
#pragma once

namespace yy {

constexpr double kPolyMaxU = 0.6;

// out of line: keeps the unrolled loops that call cubic_drift small
static __device__ __noinline__ void cubic_drift_wide(float x, float* f, float* s) { sincosf(x, s, f); }

// a * b + c on two float lanes at once (one packed FMA, each lane rounded as fmaf)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    uint64_t av, bv, cv, dv;
    asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b.x), "f"(b.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(cv) : "f"(c.x), "f"(c.y));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(dv) : "l"(av), "l"(bv), "l"(cv));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(dv));
    return d;
}
// a * b on two lanes, rounded as the float product (a packed FMA with a -0 addend, which
// leaves every product, signed zeros included, as the plain multiplication gives it)
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return ffma2(a, b, make_float2(-0.0f, -0.0f)); }

// Narrow boxes only (cc finite): the polynomial form without the fallback branch.
__device__ __forceinline__ void cubic_drift_narrow(float u, float cc, float sc, float* f, float* s) {
    const float u2 = u * u;
    const float cu =
        fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f), -0.5f), 1.0f);
    const float su =
        u * fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, 1.0f / 362880.0f, -1.0f / 5040.0f), 1.0f / 120.0f), -1.0f / 6.0f),
                 1.0f);
    *f = fmaf(cc, cu, -sc * su);
    *s = fmaf(sc, cu, cc * su);
}

// The same for two coordinates at once in packed float pairs: operation for operation the
// scalar form above, so each lane's values are bit for bit those of cubic_drift_narrow.
__device__ __forceinline__ void cubic_drift_narrow2(float2 u, float2 cc, float2 sc, float2* f, float2* s) {
    const auto k2 = [](float v) { return make_float2(v, v); };
    const float2 u2 = fmul2(u, u);
    const float2 cu = ffma2(
        u2, ffma2(u2, ffma2(u2, ffma2(u2, k2(1.0f / 40320.0f), k2(-1.0f / 720.0f)), k2(1.0f / 24.0f)), k2(-0.5f)),
        k2(1.0f));
    const float2 su = fmul2(
        u, ffma2(u2, ffma2(u2, ffma2(u2, ffma2(u2, k2(1.0f / 362880.0f), k2(-1.0f / 5040.0f)), k2(1.0f / 120.0f)),
                           k2(-1.0f / 6.0f)),
                 k2(1.0f)));
    *f = ffma2(cc, cu, fmul2(make_float2(-sc.x, -sc.y), su));
    *s = ffma2(sc, cu, fmul2(cc, su));
}

__device__ __forceinline__ void cubic_drift(float u, float hi, float lo, float cc, float sc, float* f, float* s) {
    if (cc == cc) {
        const float u2 = u * u;
        const float cu =
            fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f), -0.5f), 1.0f);
        const float su =
            u * fmaf(u2, fmaf(u2, fmaf(u2, fmaf(u2, 1.0f / 362880.0f, -1.0f / 5040.0f), 1.0f / 120.0f),
                          -1.0f / 6.0f),
                     1.0f);
        *f = fmaf(cc, cu, -sc * su);
        *s = fmaf(sc, cu, cc * su);
    } else {
        cubic_drift_wide(hi + (u + lo), f, s);
    }
}

}  // namespace yy
