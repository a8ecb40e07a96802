// Scrambled Sobol nodes on the device (Appendix A, "Sobol Sequence"; scrambling as in
// "Practical considerations" there).
//
// k_sobol_dirs: one thread per dimension turns the generator parameters (primitive
// polynomial x^s + a_1 x^{s-1} + ... + a_{s-1} x + 1 and initial m_1..m_s) into the 32
// direction integers V_k = m_k 2^{32-k}, continued for k > s by
//     V_k = V_{k-s} ^ (V_{k-s} >> s) ^ XOR_{i<s, a_i = 1} V_{k-i},
// and pre-multiplies them by the scramble matrix (the scramble y -> L y ^ e is linear in
// the XOR of direction integers, so L can be applied once per direction integer).
//
// k_sobol_points: thread per (point, dimension): XOR of the scrambled direction integers
// selected by the Gray code g = i ^ (i >> 1), XOR the digital shift, then the box map
// u = R (2 (y + 1/2) 2^-32 - 1) in float64 with explicit round-to-nearest operations
// (no contraction), rounded once more to float32.
#include "yy_internal.cuh"

namespace yy {

__global__ void k_sobol_dirs(const uint32_t* __restrict__ params, uint32_t* __restrict__ dirs,
                             int r) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= r) return;
    const uint32_t* p = params + (size_t)d * (YY_SOBOL_POLY_WORDS + YY_SOBOL_SCRAMBLE_WORDS);
    const uint32_t* L = p + YY_SOBOL_POLY_WORDS;
    uint32_t V[33];
    const int s = (int)p[0];
    const uint32_t a = p[1];
    if (s == 0) {
        for (int k = 1; k <= 32; ++k) V[k] = 1u << (32 - k);
    } else {
        for (int k = 1; k <= s && k <= 32; ++k) V[k] = p[1 + k] << (32 - k);
        for (int k = s + 1; k <= 32; ++k) {
            uint32_t v = V[k - s] ^ (V[k - s] >> s);
            for (int i = 1; i < s; ++i)
                if ((a >> (s - 1 - i)) & 1u) v ^= V[k - i];
            V[k] = v;
        }
    }
    uint32_t* out = dirs + (size_t)d * 33;
    for (int b = 1; b <= 32; ++b) {
        uint32_t w = 0;
        for (int k = 1; k <= 32; ++k) w |= (uint32_t)(__popc(L[k - 1] & V[b]) & 1) << (32 - k);
        out[b - 1] = w;
    }
    out[32] = L[32];
}

__global__ void k_sobol_points(const uint32_t* __restrict__ dirs, int r, int r_pad,
                               long long first, long long count, float* __restrict__ u,
                               uint32_t* __restrict__ bits, const double* __restrict__ halfwidth) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= r) return;
    const uint32_t* V = dirs + (size_t)d * 33;
    const double R = halfwidth ? halfwidth[d] : 0.0;
    for (long long i = blockIdx.y * (long long)blockDim.y + threadIdx.y; i < count;
         i += (long long)gridDim.y * blockDim.y) {
        const unsigned long long idx = (unsigned long long)(first + i);
        const uint32_t g = (uint32_t)(idx ^ (idx >> 1));
        uint32_t y = V[32];
#pragma unroll 8
        for (int b = 0; b < 32; ++b)
            if ((g >> b) & 1u) y ^= V[b];
        if (bits) bits[(size_t)i * r + d] = y;
        if (u) {
            double t = __dadd_rn((double)y, 0.5);
            t = __dmul_rn(t, 0x1p-31);      // 2 (y + 1/2) 2^-32, exact
            t = __dsub_rn(t, 1.0);          // exact
            u[(size_t)(first + i) * r_pad + d] = __double2float_rn(__dmul_rn(R, t));
        }
    }
}

// Re-mapping of the reference nodes to new half-widths during a restart (no-op unless the
// restart flag and the scale-changed flag are set).
__global__ void k_sobol_points_restart(const uint32_t* __restrict__ dirs, int r, int r_pad, long long n,
                                       float* __restrict__ u, const double* __restrict__ half,
                                       const DevStats* __restrict__ st) {
    if (st->restart_flag == 0 || st->scale_changed == 0) return;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= r) return;
    const uint32_t* V = dirs + (size_t)d * 33;
    const double R = half[d];
    for (long long i = blockIdx.y * (long long)blockDim.y + threadIdx.y; i < n; i += (long long)gridDim.y * blockDim.y) {
        const unsigned long long idx = (unsigned long long)i;
        const uint32_t g = (uint32_t)(idx ^ (idx >> 1));
        uint32_t y = V[32];
#pragma unroll 8
        for (int b = 0; b < 32; ++b)
            if ((g >> b) & 1u) y ^= V[b];
        double t = __dadd_rn((double)y, 0.5);
        t = __dmul_rn(t, 0x1p-31);
        t = __dsub_rn(t, 1.0);
        u[(size_t)i * r_pad + d] = __double2float_rn(__dmul_rn(R, t));
    }
}

// Halton and Faure nodes (Appendix A, "Halton Sequence" and "Faure Sequence"): thread per
// (point, dimension), index k = first + i.  The fraction's base-p digits y_0, y_1, ... (most
// significant first) form the integer R = sum_i y_i p^(M-1-i) with M the largest digit count
// such that p^M <= 2^53, so R and p^M are exact in float64 and R / p^M is the correctly
// rounded fraction whatever M is.
//   Halton: p = the d-th prime, y_i = digit i of k (least significant first): the radical
//           inverse.
//   Faure:  p = the smallest prime >= r, y = C k mod p with C = P^(d-1), P_ij = binom(j, i);
//           the power of the Pascal matrix has the closed form
//           (P^c)_ij = binom(j, i) c^(j-i), used here (c = d - 1 mod p).
// Box map as for Sobol nodes: u = R_d (2 phi - 1), float64 with explicit rounding, then float32.
__device__ __forceinline__ int lds_digits(unsigned long long p, unsigned long long* pM) {
    int M = 0;
    unsigned long long v = 1;
    while (v <= (1ull << 53) / p) { v *= p; ++M; }
    *pM = v;
    return M;
}

__global__ void k_lds_points(int kind, const uint32_t* __restrict__ primes, uint32_t p_faure, int r, int r_pad,
                             long long first, long long count, float* __restrict__ u,
                             const double* __restrict__ halfwidth) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= r) return;
    const unsigned long long p = (kind == YY_NODES_HALTON) ? primes[d] : p_faure;
    unsigned long long pM;
    const int M = lds_digits(p, &pM);
    const double R = halfwidth[d];
    const unsigned long long c = (unsigned long long)d % p;   // Faure: power of the Pascal matrix
    unsigned long long cp[64];                                  // c^t mod p
    if (kind == YY_NODES_FAURE) {
        cp[0] = 1 % p;
        for (int t = 1; t < M; ++t) cp[t] = (cp[t - 1] * c) % p;
    }
    for (long long i = blockIdx.y * (long long)blockDim.y + threadIdx.y; i < count; i += (long long)gridDim.y * blockDim.y) {
        unsigned long long kk = (unsigned long long)(first + i);
        unsigned long long dig[64];
        for (int t = 0; t < M; ++t) { dig[t] = kk % p; kk /= p; }
        unsigned long long Rn = 0;
        for (int a = 0; a < M; ++a) {
            unsigned long long y;
            if (kind == YY_NODES_HALTON) {
                y = dig[a];
            } else {
                // y_a = sum_{j >= a} binom(j, a) c^(j-a) k_j mod p
                unsigned long long acc = 0, binom = 1;   // binom(j, a), starting at j = a
                for (int j = a; j < M; ++j) {
                    if (j > a) binom = binom * (unsigned long long)j / (unsigned long long)(j - a);
                    acc += ((binom % p) * cp[j - a] % p) * dig[j];
                }
                y = acc % p;
            }
            Rn = Rn * p + y;
        }
        const double phi = __ddiv_rn((double)Rn, (double)pM);
        const double t = __dsub_rn(__dmul_rn(2.0, phi), 1.0);
        u[(size_t)i * r_pad + d] = __double2float_rn(__dmul_rn(R, t));
    }
}

cudaError_t launch_lds_points(int kind, const uint32_t* primes, uint32_t p_faure, int r, int r_pad, long long n,
                              float* u, const double* halfwidth, cudaStream_t s) {
    dim3 block(64, 4);
    long long gy = (n + 3) / 4;
    if (gy > 65535) gy = 65535;
    k_lds_points<<<dim3((r + 63) / 64, (unsigned)gy), block, 0, s>>>(kind, primes, p_faure, r, r_pad, 1, n, u, halfwidth);
    return cudaGetLastError();
}

cudaError_t launch_sobol_points_restart(const uint32_t* dirs, int r, int r_pad, long long n, float* u,
                                        const double* next_half, const DevStats* st, cudaStream_t s) {
    dim3 block(64, 4);
    long long gy = (n + 3) / 4;
    if (gy > 65535) gy = 65535;
    k_sobol_points_restart<<<dim3((r + 63) / 64, (unsigned)gy), block, 0, s>>>(dirs, r, r_pad, n, u, next_half, st);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sobol_dirs(const uint32_t* params, uint32_t* dirs, int r, cudaStream_t s) {
    k_sobol_dirs<<<(r + 63) / 64, 64, 0, s>>>(params, dirs, r);
    return cudaGetLastError();
}
template cudaError_t launch_sobol_dirs<float>(const uint32_t*, uint32_t*, int, cudaStream_t);
template cudaError_t launch_sobol_dirs<double>(const uint32_t*, uint32_t*, int, cudaStream_t);

cudaError_t launch_sobol_points(const uint32_t* dirs, int r, int r_pad, long long first,
                                long long count, float* u, uint32_t* bits, const double* halfwidth,
                                cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    dim3 block(64, 4);
    long long gy = (count + 3) / 4;
    if (gy > 65535) gy = 65535;
    dim3 grid((r + 63) / 64, (unsigned)gy);
    k_sobol_points<<<grid, block, 0, s>>>(dirs, r, r_pad, first, count, u, bits, halfwidth);
    return cudaGetLastError();
}

}  // namespace yy
