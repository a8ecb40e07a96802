// Per-target combination of the N kernel terms with the identity term of eq.
// general_kernel ("High-Order Kernel Construction"), in log space, relative to c_ref:
//   ell_pred(i) - c_ref = log( sum_j c_j e^{L_j(i) - c_ref} + c_{N+1} e^{ell(i) - c_ref} ),
//   L_j(i) - c_ref = (C_j - c_ref) - tau_j div f(x_i) - hld_i + m_j + log s_j,
// where (m_j, s_j) is the online log-sum-exp state of the scaled kernel scores over the
// sources and hld_i = 1/2 log det_+ a(x_i) with noise coefficients (0 for unit noise).  Signed log-sum-exp: a non-positive total gives -inf and is counted.
#pragma once

#include "yy_internal.cuh"

namespace yy {

template <typename T> __device__ __forceinline__ T cmb_exp(T x);
template <> __device__ __forceinline__ float cmb_exp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double cmb_exp<double>(double x) { return exp(x); }
template <typename T> __device__ __forceinline__ T cmb_log(T x);
template <> __device__ __forceinline__ float cmb_log<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double cmb_log<double>(double x) { return log(x); }

template <typename T, int N>
__device__ __forceinline__ T combine_scales(const Consts<T>& k, const T (&mx)[N], const T (&sm)[N],
                                            T divf, T logw_i, double c_ref, unsigned int* clamps, T hld = T(0)) {
    T term[N + 1], sg[N + 1];
    T M = T(-INFINITY);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const T L = (mx[j] == T(-INFINITY)) ? T(-INFINITY)
                                            : k.cj_off[j] - k.tau[j] * divf - hld + mx[j] + cmb_log<T>(sm[j]);
        sg[j] = k.sign_c[j];
        term[j] = (sg[j] == T(0) || L == T(-INFINITY)) ? T(-INFINITY) : k.logabs_c[j] + L;
        M = fmax(M, term[j]);
    }
    sg[N] = k.sign_c[N];
    term[N] = (sg[N] == T(0) || logw_i == T(-INFINITY))
                  ? T(-INFINITY)
                  : k.logabs_c[N] + (T)((double)logw_i - c_ref);
    M = fmax(M, term[N]);
    if (M == T(-INFINITY)) return T(-INFINITY);
    T S = T(0);
#pragma unroll
    for (int j = 0; j <= N; ++j)
        if (term[j] != T(-INFINITY)) S += sg[j] * cmb_exp<T>(term[j] - M);
    if (S > T(0)) return M + cmb_log<T>(S);
    atomicAdd(clamps, 1u);
    return T(-INFINITY);
}

}  // namespace yy
