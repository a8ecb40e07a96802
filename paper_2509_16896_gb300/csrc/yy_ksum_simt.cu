// Prediction step, plain form on the FMA pipes (float32 or float64).
//
// For every target i and scale j (tau_j = dt / 2^(j-1)), in units relative to c_ref:
//   L_j(i) - c_ref = (C_j - c_ref) - tau_j div f(x_i)
//                    + LSE_s [ -|u_i - tau_j f_i - u_s|^2 / (2 tau_j) + ell_s ],
//   C_j = -(r/2) log(2 pi tau_j) + log w_q,
// which is log sum_s K_{tau_j}(x_i, x_s) w_q e^{ell_s} for the first-order kernel of
// eq. kernel ("First-Order Kernel Construction") after completing the square:
//   -|x-y|^2/(2 tau) - (y-x).f(x) - tau(div f + |f|^2/2) = -|x - tau f(x) - y|^2/(2 tau) - tau div f.
// Differences are formed first: with D = u_i - u_s, S1 = |D|^2 and S2 = D.f_i,
//   |u_i - tau f_i - u_s|^2 = S1 - 2 tau S2 + tau^2 |f_i|^2,
// so one pass over the coordinates serves all N scales.  The N terms are combined with
// the identity term of eq. general_kernel by a signed log-sum-exp; a non-positive total
// gives -inf (counted).
//
// Tiling: a CTA owns 64 targets and sweeps all sources in tiles of 64, staging 16
// coordinates of the target rows, their drift and the source rows in shared memory per
// step; each of the 256 threads holds a 4x4 block of (S1, S2) accumulators and, per
// target and scale, an online (max, sum) of the exponentials, merged across the 16
// threads of a target group at the end.
#include <algorithm>

#include "yy_combine.cuh"
#include "yy_tcgen05.cuh"

namespace yy {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;

template <typename T> __device__ __forceinline__ T exp_fast(T x);
template <> __device__ __forceinline__ float exp_fast<float>(float x) { return exp2f(x * 1.4426950408889634f); }
template <> __device__ __forceinline__ double exp_fast<double>(double x) { return exp(x); }
}  // namespace

// SCREEN (float32 only): before a source tile is evaluated, the squared distance of each
// of its pairs over the first k1 coordinates -- a lower bound of the full |u_i - u_s|^2 --
// is bounded from below through its Gram form q_i + q_s - 2 G (q the norms over those
// coordinates from the preparation pass, G = sum u_i u_s by one FMA per coordinate), less
// the rounding allowance 3 gamma_k1 (q_i + q_s) of the FMA chain (gamma_k = k 2^-24 /
// (1 - k 2^-24); 2 |u_i||u_s| <= q_i + q_s) and 1e-5 (q_i + q_s) for the norms' own
// rounding, and compared with rho_i^2, where
//     rho_i = max_j [tau_j |f_i| + sqrt(2 tau_j max(0, lmax - (ell_i - tau_j |f_i|^2 / 2) + T))],
// lmax the largest live source log-weight, ell_i - tau_j |f_i|^2 / 2 the exact self term of
// row i (a lower bound of its largest term) and T = ln n + 20.  By the triangle inequality
// |u_i - tau_j f_i - u_s| >= |u_i - u_s| - tau_j |f_i|, a pair beyond rho_i scores below the
// self term by more than T at every scale, so a tile none of whose live pairs passes is
// skipped (all skipped terms together are below e^-20 of the row's sum); any other tile is
// evaluated exactly as in the plain form.  A live target without a finite log-weight has no
// reference and takes every tile.  The comparison carries a relative margin of 1e-4 for
// the float32 rounding of the partial sums.
// NOISE (diagonal noise coefficients): the squared distance and the drift's inner product
// take the target's metric a(x_i)^+, S1 = sum_d m_d D_d^2, S2 = sum_d m_d D_d f_d, with
// |f_i|^2 in the same metric (nf) and -1/2 log det_+ a(x_i) added in the combination.
// OPBUILD (float32): the materialised operator -- every pair's score without the source
// weight, A_j(i, s) = -S1 / (2 tau_j) + S2 - tau_j |f_i|^2 / 2, is written to b.op instead of
// being accumulated.
// split / nsplit (plain form of a filter with few target blocks): this block sweeps only the
// split-th of nsplit equal ranges of source tiles and stores its rows' partial (max, sum)
// per scale in b.simt_part; k_simt_merge combines the ranges.
template <typename T, int N, bool SCREEN = false, bool NOISE = false, bool OPBUILD = false>
__device__ __forceinline__ void ksum_simt_body(const Consts<T>& k, const Bufs<T>& b, int rk, int bid, int k1 = 0,
                                               int split = 0, int nsplit = 1) {
    __shared__ T At[BK][BM];   // u of targets
    __shared__ T Ft[BK][BM];   // f of targets
    __shared__ T Bt[BK][BN];   // u of sources
    __shared__ T Mt[NOISE ? BK : 1][NOISE ? BM : 1];   // metric of targets
    __shared__ T lsrc[BN];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const long long i0 = (long long)bid * BM;

    T rowc[TM][N];          // -(tau_j / 2) |f_i|^2
    T mx[TM][N], sm[TM][N];
    T rho2[TM];             // SCREEN: squared screening radius of each row
    T q1t[TM];              // SCREEN: first-pass norms of the target rows
    __shared__ T q1s[SCREEN ? BN : 1];   // SCREEN: first-pass norms of the tile's sources
    const T gam = SCREEN ? T(3.03) * (T)k1 * T(5.9604645e-8) + T(1e-5) : T(0);   // rounding allowance per (q_i + q_s)
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        const long long i = i0 + ty * TM + a;
        const T nf = (i < k.n) ? b.nf[i] : T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            rowc[a][j] = -T(0.5) * k.tau[j] * nf;
            mx[a][j] = T(-INFINITY);
            sm[a][j] = T(0);
        }
        rho2[a] = T(-1);   // no candidates (padded or masked rows)
        if constexpr (SCREEN) {   // first-pass norm of the target row
            q1t[a] = T(0);
            if (i < k.n)
                for (int c = 0; c < k1 / 64; ++c) q1t[a] += b.nu_chunk[(size_t)i * (k.r_pad / 64) + c];
        }
        if constexpr (SCREEN) {
            if (i < k.n && !b.mask[i]) {
                const T li = b.logw[i];
                const T lmax = (T)b.stats->scr_lmax;
                if (li == T(-INFINITY)) {
                    rho2[a] = T(INFINITY);
                } else {
                    const T Tn = log((T)k.n) + T(20);
                    const T Fi = sqrt(nf);
                    T rho = T(0);
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        const T gap = fmax(lmax - (rowc[a][j] + li) + Tn, T(0));
                        rho = fmax(rho, k.tau[j] * Fi + sqrt(T(2) * k.tau[j] * gap));
                    }
                    rho2[a] = rho * rho * T(1.0001) + T(1e-30);
                }
            }
        }
    }

    const long long src_tiles = (k.n + BN - 1) / BN;
    const long long s_begin = (src_tiles * split / nsplit) * BN;
    const long long s_end = std::min<long long>(k.n, (src_tiles * (split + 1) / nsplit) * BN);
    for (long long s0 = s_begin; s0 < s_end; s0 += BN) {
        T S1[TM][TN], S2[TM][TN];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int c = 0; c < TN; ++c) { S1[a][c] = T(0); S2[a][c] = T(0); }
        if (tid < BN) {
            const long long s = s0 + tid;
            lsrc[tid] = (s < k.n && !b.mask[s]) ? b.logw[s] : T(-INFINITY);
            if constexpr (SCREEN) {
                T q = T(0);
                if (s < k.n)
                    for (int c = 0; c < k1 / 64; ++c) q += b.nu_chunk[(size_t)s * (k.r_pad / 64) + c];
                q1s[tid] = q;
            }
        }
        if constexpr (SCREEN) {
            // first pass: Gram products G over coordinates [0, k1)
            for (int d0 = 0; d0 < k1; d0 += BK) {
                __syncthreads();
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int e = tid + 256 * q;
                    const int row = e >> 4, col = e & 15;
                    At[col][row] = (T)b.u[(size_t)(i0 + row) * k.r_pad + d0 + col];
                    Bt[col][row] = (T)b.u[(size_t)(s0 + row) * k.r_pad + d0 + col];
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    T av[TM], bv[TN];
#pragma unroll
                    for (int a = 0; a < TM; ++a) av[a] = At[kk][ty * TM + a];
#pragma unroll
                    for (int c = 0; c < TN; ++c) bv[c] = Bt[kk][tx * TN + c];
#pragma unroll
                    for (int a = 0; a < TM; ++a)
#pragma unroll
                        for (int c = 0; c < TN; ++c) S1[a][c] = fma(av[a], bv[c], S1[a][c]);
                }
            }
            int any = 0;
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int c = 0; c < TN; ++c) {
                    const T qq = q1t[a] + q1s[tx * TN + c];
                    const T lower = qq - T(2) * S1[a][c] - gam * qq;   // lower bound of the partial |u_i - u_s|^2
                    any |= (lower <= rho2[a] && lsrc[tx * TN + c] != T(-INFINITY)) ? 1 : 0;
                }
            if (!__syncthreads_or(any)) continue;   // every pair of the tile is negligible
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int c = 0; c < TN; ++c) S1[a][c] = T(0);
        }
        for (int d0 = 0; d0 < rk; d0 += BK) {
            __syncthreads();
            // 64 rows x 16 coordinates per operand; 256 threads x 4 values
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = tid + 256 * q;
                const int row = e >> 4, col = e & 15;
                const size_t ti = (size_t)(i0 + row) * k.r_pad + d0 + col;
                const size_t si = (size_t)(s0 + row) * k.r_pad + d0 + col;
                At[col][row] = (T)b.u[ti];
                Ft[col][row] = b.f[ti];
                Bt[col][row] = (T)b.u[si];
                if constexpr (NOISE) Mt[col][row] = b.minv[ti];
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T av[TM], fv[TM], bv[TN], mv[TM];
#pragma unroll
                for (int a = 0; a < TM; ++a) { av[a] = At[kk][ty * TM + a]; fv[a] = Ft[kk][ty * TM + a]; }
                if constexpr (NOISE) {
#pragma unroll
                    for (int a = 0; a < TM; ++a) { mv[a] = Mt[kk][ty * TM + a]; fv[a] *= mv[a]; }
                }
#pragma unroll
                for (int c = 0; c < TN; ++c) bv[c] = Bt[kk][tx * TN + c];
#pragma unroll
                for (int a = 0; a < TM; ++a)
#pragma unroll
                    for (int c = 0; c < TN; ++c) {
                        const T dlt = av[a] - bv[c];
                        if constexpr (NOISE) S1[a][c] = fma(mv[a] * dlt, dlt, S1[a][c]);
                        else S1[a][c] = fma(dlt, dlt, S1[a][c]);
                        S2[a][c] = fma(dlt, fv[a], S2[a][c]);
                    }
            }
        }
        if constexpr (OPBUILD) {
            const size_t plane = (size_t)k.n_pad * (size_t)k.n_pad;
#pragma unroll
            for (int a = 0; a < TM; ++a) {
                const long long i = i0 + ty * TM + a;
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    float4 v;
                    v.x = (float)(fma(-S1[a][0], k.inv2tau[j], S2[a][0]) + rowc[a][j]);
                    v.y = (float)(fma(-S1[a][1], k.inv2tau[j], S2[a][1]) + rowc[a][j]);
                    v.z = (float)(fma(-S1[a][2], k.inv2tau[j], S2[a][2]) + rowc[a][j]);
                    v.w = (float)(fma(-S1[a][3], k.inv2tau[j], S2[a][3]) + rowc[a][j]);
                    *reinterpret_cast<float4*>(b.op + j * plane + (size_t)i * k.n_pad + s0 + tx * TN) = v;
                }
            }
            __syncthreads();
            continue;
        }
        // scores and online log-sum-exp for this source tile
        T ls[TN];
#pragma unroll
        for (int c = 0; c < TN; ++c) ls[c] = lsrc[tx * TN + c];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
            for (int j = 0; j < N; ++j) {
                T sc[TN];
                T tmax = T(-INFINITY);
#pragma unroll
                for (int c = 0; c < TN; ++c) {
                    sc[c] = fma(-S1[a][c], k.inv2tau[j], S2[a][c]) + (rowc[a][j] + ls[c]);
                    tmax = fmax(tmax, sc[c]);
                }
                if (tmax == T(-INFINITY)) continue;
                if (tmax > mx[a][j]) {
                    sm[a][j] = (mx[a][j] == T(-INFINITY)) ? T(0) : sm[a][j] * exp_fast<T>(mx[a][j] - tmax);
                    mx[a][j] = tmax;
                }
#pragma unroll
                for (int c = 0; c < TN; ++c) sm[a][j] += exp_fast<T>(sc[c] - mx[a][j]);
            }
        __syncthreads();
    }

    if constexpr (OPBUILD) return;
    // merge the 16 threads that share a target group (lanes differing in the low 4 bits)
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            T m = mx[a][j], s = sm[a][j];
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                const T m2 = __shfl_xor_sync(0xffffffffu, m, o);
                const T s2 = __shfl_xor_sync(0xffffffffu, s, o);
                if (m2 != T(-INFINITY)) {
                    if (m == T(-INFINITY)) { m = m2; s = s2; }
                    else if (m2 > m) { s = s * exp_fast<T>(m - m2) + s2; m = m2; }
                    else { s += s2 * exp_fast<T>(m2 - m); }
                }
            }
            mx[a][j] = m;
            sm[a][j] = s;
        }
    if (tx != 0) return;
    if (nsplit > 1) {   // this range's states; the merge applies the combination
#pragma unroll
        for (int a = 0; a < TM; ++a) {
            const long long i = i0 + ty * TM + a;
            if (i >= k.n) continue;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                T* ps = b.simt_part + (((size_t)i * kSimtMaxSplit + split) * kMaxScales + j) * 2;
                ps[0] = mx[a][j];
                ps[1] = sm[a][j];
            }
        }
        return;
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        const long long i = i0 + ty * TM + a;
        if (i >= k.n) continue;
        if (b.mask[i]) { b.logw_pred[i] = T(-INFINITY); continue; }
        const T hld = NOISE ? b.hld[i] : T(0);
        b.logw_pred[i] = combine_scales<T, N>(k, mx[a], sm[a], b.divf[i], b.logw[i], b.stats->c_ref, &b.stats->clamps,
                                              hld);
    }
}

template <typename T, int N, bool NOISE = false>
__global__ void __launch_bounds__(256) k_ksum_simt(Consts<T> k, Bufs<T> b, int rk, int nsplit) {
    ksum_simt_body<T, N, false, NOISE>(k, b, rk, (int)(k.row0 / BM) + (int)(blockIdx.x / nsplit), 0,
                                       (int)(blockIdx.x % nsplit), nsplit);
}

// Merges the source ranges' (max, sum) states of every row and applies the multi-scale
// combination (the plain form with nsplit > 1).
template <typename T, int N, bool NOISE = false>
__global__ void __launch_bounds__(256) k_simt_merge(Consts<T> k, Bufs<T> b, int nsplit) {
    const long long i = k.row0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k.row1 || i >= k.n) return;
    if (b.mask[i]) { b.logw_pred[i] = T(-INFINITY); return; }
    T mx[N], sm[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        T m = T(-INFINITY), s = T(0);
        for (int q = 0; q < nsplit; ++q) {
            const T* ps = b.simt_part + (((size_t)i * kSimtMaxSplit + q) * kMaxScales + j) * 2;
            const T m2 = ps[0], s2 = ps[1];
            if (m2 == T(-INFINITY)) continue;
            if (m == T(-INFINITY)) { m = m2; s = s2; }
            else if (m2 > m) { s = s * exp_fast<T>(m - m2) + s2; m = m2; }
            else { s += s2 * exp_fast<T>(m2 - m); }
        }
        mx[j] = m;
        sm[j] = s;
    }
    const T hld = NOISE ? b.hld[i] : T(0);
    b.logw_pred[i] = combine_scales<T, N>(k, mx, sm, b.divf[i], b.logw[i], b.stats->c_ref, &b.stats->clamps, hld);
}

template <int N>
__global__ void __launch_bounds__(256) k_ksum_scr32(Consts<float> k, Bufs<float> b, int rk, int k1) {
    ksum_simt_body<float, N, true>(k, b, rk, (int)(k.row0 / BM) + blockIdx.x, k1);
}

// Materialised operator: built only when the node set moved since the last build (the flag
// is set by restarts and state changes, cleared by the apply), unless forced.
template <int N>
__global__ void __launch_bounds__(256) k_op_build(Consts<float> k, Bufs<float> b, int rk, int force) {
    if (!force && b.stats->op_stale == 0) return;
    ksum_simt_body<float, N, false, false, true>(k, b, rk, (int)(k.row0 / BM) + blockIdx.x);
}

// The apply works in base 2: with v = A + ell, e^(v - m) = 2^(v log2 e - m log2 e).
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// 2^x by the hardware approximation (PTX ex2.approx.ftz.f32): its results below 2^-126 are
// flushed to zero, which here are terms below 2^-126 of the running maximum.
__device__ __forceinline__ float ex2_hw(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// No term yet: a finite stand-in for -inf in the apply's running maxima, so that
// 2^(v - m) and the merges need no test (2^(-inf - kOpNone) = 0, 2^(kOpNone - v) = 0 for
// any score v the operator can produce, 2^(kOpNone - kOpNone) = 1 with both sums zero).
constexpr float kOpNone = -3.402823466e38f;

// Source terms of the apply in base 2: log2 e ell_s for live sources, -inf for masked nodes
// and for the padding beyond n.
__global__ void __launch_bounds__(256) k_op_src(Consts<float> k, Bufs<float> b) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= k.n_pad) return;
    b.op_lsrc[s] = (s < k.n && !b.mask[s]) ? b.logw[s] * kLog2e : -INFINITY;
}

// Online base-2 (max, sum) over four scores A log2 e + l.  Every streamed operator entry
// is finite (the build writes whole 64-column source tiles of the zero-initialised
// workspace), so a -inf source term gives a -inf score.  One rescale per group of four
// when its largest score is a new maximum.
__device__ __forceinline__ void op_lse4(float& m, float& s, const float4 a, const float4 l) {
    const float v0 = fmaf(a.x, kLog2e, l.x), v1 = fmaf(a.y, kLog2e, l.y);
    const float v2 = fmaf(a.z, kLog2e, l.z), v3 = fmaf(a.w, kLog2e, l.w);
    const float vm = fmaxf(fmaxf(v0, v1), fmaxf(v2, v3));
    if (vm > m) { s *= ex2_hw(m - vm); m = vm; }
    s += (ex2_hw(v0 - m) + ex2_hw(v1 - m)) + (ex2_hw(v2 - m) + ex2_hw(v3 - m));
}

// Merge of two base-2 (max, sum) states.
__device__ __forceinline__ void op_merge(float& m, float& s, float m2, float s2) {
    const float mm = fmaxf(m, m2);
    s = s * ex2_hw(m - mm) + s2 * ex2_hw(m2 - mm);
    m = mm;
}

namespace {
constexpr int kOpCW = 2048;   // columns of one plane in a stage of the apply's ring
constexpr unsigned long long kOpDrainNs = 4000000000ull;   // bound of the exit drain (4 s)
template <int N> constexpr int op_stages() { return 8 / N > 2 ? 8 / N : 2; }
template <int N> constexpr size_t op_smem_bytes() {
    return (size_t)op_stages<N>() * N * kOpCW * sizeof(float) + 2 * op_stages<N>() * sizeof(uint64_t);
}
// Untiled bulk copy global -> shared (both addresses 16-byte aligned, size a multiple of
// 16) completing on an mbarrier.
__device__ __forceinline__ void op_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    uint64_t g;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(reinterpret_cast<uint64_t>(src)));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     ptx::smem_u32(dst)),
                 "l"(g), "r"(bytes), "r"(ptx::smem_u32(bar))
                 : "memory");
}
// Wait for a phase, bounded by limit_ns: on expiry the block's abort flag and the status
// word's timeout bit are set; a raised abort flag ends the wait as well.
__device__ __forceinline__ bool op_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                        unsigned int* status, unsigned long long limit_ns) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = ptx::globaltimer();
    while (true) {
        if (ptx::mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (ptx::globaltimer() - t0 > limit_ns) {
            *abort_flag = 1;
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
}
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
}  // namespace

// L_j(i) = log sum_s exp(A_j(i, s) + ell_s) over live sources, then the signed combination
// of the scales with the identity term.  A block owns one target row at a time (rows are
// strided over the grid, so every block gets the same share).  Warp 8 streams the row's N
// planes through a ring of shared-memory stages with bulk async copies (kOpCW columns of
// every plane per stage); warps 0-7 take float4 groups of each stage, keep an online base-2
// (max, sum) per scale, release the stage, and merge their 256 states at the end of the
// row.  Every wait is bounded by the handle's limit; after a timeout the consumers keep
// the same barrier sequence without computing, and the producer waits (bounded) for its
// copies in flight before it exits.
template <int N>
__global__ void __launch_bounds__(288) k_op_apply(Consts<float> k, Bufs<float> b) {
    constexpr int S = op_stages<N>();
    extern __shared__ __align__(128) unsigned char op_smem[];
    float* stage = reinterpret_cast<float*>(op_smem);
    uint64_t* full = reinterpret_cast<uint64_t*>(op_smem + (size_t)S * N * kOpCW * sizeof(float));
    uint64_t* empty = full + S;
    __shared__ float red_m[2][N][8], red_s[2][N][8];
    __shared__ int abort_flag;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            ptx::mbar_init(&full[q], 1);
            ptx::mbar_init(&empty[q], 8);
        }
        ptx::mbar_fence_init();
        abort_flag = 0;
        if (blockIdx.x == 0) b.stats->op_stale = 0;
    }
    __syncthreads();
    volatile int* ab = &abort_flag;
    unsigned int* status = &b.stats->status;
    const long long n4 = (k.n + 3) / 4 * 4;   // columns streamed per row: a multiple of 16 bytes
    const int chunks = (int)((n4 + kOpCW - 1) / kOpCW);
    const size_t plane = (size_t)k.n_pad * (size_t)k.n_pad;
    const float4* lsrc = reinterpret_cast<const float4*>(b.op_lsrc);

    if (wid == 8) {   // producer
        if (lane != 0) return;
        uint32_t it = 0;
        for (long long i = k.row0 + blockIdx.x; i < k.row1 && !*ab; i += gridDim.x) {
            for (int c = 0; c < chunks; ++c) {
                const uint32_t slot = it % S, ph = (it / S) & 1u;
                if (!op_wait(&empty[slot], ph ^ 1u, ab, status, k.wait_ns)) break;
                const long long c0 = (long long)c * kOpCW;
                const uint32_t bytes = (uint32_t)((n4 - c0 < kOpCW ? n4 - c0 : kOpCW) * sizeof(float));
                ptx::mbar_arrive_expect_tx(&full[slot], N * bytes);
#pragma unroll
                for (int j = 0; j < N; ++j)
                    op_bulk_load(stage + ((size_t)slot * N + j) * kOpCW, b.op + j * plane + (size_t)i * k.n_pad + c0,
                                 bytes, &full[slot]);
                ++it;
            }
        }
        // the last S stages issued have landed before the block's shared memory is released
        for (uint32_t t = it > (uint32_t)S ? it - S : 0u; t < it; ++t) {
            const unsigned long long t0 = ptx::globaltimer();
            while (!ptx::mbar_try_wait(&full[t % S], (t / S) & 1u))
                if (ptx::globaltimer() - t0 > kOpDrainNs) break;
        }
        return;
    }

    uint32_t it = 0;
    int par = 0;
    for (long long i = k.row0 + blockIdx.x; i < k.row1; i += gridDim.x, par ^= 1) {
        float m[N], s[N];
#pragma unroll
        for (int j = 0; j < N; ++j) { m[j] = kOpNone; s[j] = 0.f; }
        for (int c = 0; c < chunks; ++c, ++it) {
            const uint32_t slot = it % S, ph = (it / S) & 1u;
            if (!*ab && op_wait(&full[slot], ph, ab, status, k.wait_ns)) {
                const long long g0 = (long long)c * (kOpCW / 4);
                const int groups = (int)((n4 / 4 - g0) < kOpCW / 4 ? (n4 / 4 - g0) : kOpCW / 4);
                const float4* st = reinterpret_cast<const float4*>(stage + (size_t)slot * N * kOpCW);
                if (groups == kOpCW / 4) {   // a full stage: two groups per thread
                    const float4 l0 = __ldg(lsrc + g0 + tid), l1 = __ldg(lsrc + g0 + tid + 256);
                    float4 a0[N], a1[N];
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        a0[j] = st[j * (kOpCW / 4) + tid];
                        a1[j] = st[j * (kOpCW / 4) + tid + 256];
                    }
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        op_lse4(m[j], s[j], a0[j], l0);
                        op_lse4(m[j], s[j], a1[j], l1);
                    }
                } else {
                    for (int g = tid; g < groups; g += 256) {
                        const float4 l = __ldg(lsrc + g0 + g);
#pragma unroll
                        for (int j = 0; j < N; ++j) op_lse4(m[j], s[j], st[j * (kOpCW / 4) + g], l);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[slot]);
        }
#pragma unroll
        for (int j = 0; j < N; ++j) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                op_merge(m[j], s[j], __shfl_xor_sync(0xffffffffu, m[j], o), __shfl_xor_sync(0xffffffffu, s[j], o));
            if (lane == 0) { red_m[par][j][wid] = m[j]; red_s[par][j][wid] = s[j]; }
        }
        // One barrier of the 8 consumer warps per row: the next row writes the other parity,
        // and a row two ahead writes this one only after the next row's barrier, which warp 0
        // reaches after reading this row's states.
        consumer_sync();
        if (wid == 0 && !*ab) {
#pragma unroll
            for (int j = 0; j < N; ++j) {
                m[j] = lane < 8 ? red_m[par][j][lane] : kOpNone;
                s[j] = lane < 8 ? red_s[par][j][lane] : 0.f;
#pragma unroll
                for (int o = 4; o > 0; o >>= 1)
                    op_merge(m[j], s[j], __shfl_xor_sync(0xffffffffu, m[j], o), __shfl_xor_sync(0xffffffffu, s[j], o));
                m[j] = m[j] == kOpNone ? -INFINITY : m[j] * kLn2;   // natural log of the row's largest term
            }
            if (lane == 0)
                b.logw_pred[i] = b.mask[i] ? -INFINITY
                                           : combine_scales<float, N>(k, m, s, b.divf[i], b.logw[i], b.stats->c_ref,
                                                                      &b.stats->clamps);
        }
    }
}

cudaError_t launch_op_build(const Consts<float>& k, const Bufs<float>& b, bool force, cudaStream_t s) {
    if (!b.op) return cudaErrorInvalidValue;
    const int rk = ((k.r + BK - 1) / BK) * BK;
    const unsigned grid = (unsigned)((k.row1 - k.row0 + BM - 1) / BM);
    if (grid == 0) return cudaSuccess;
    switch (k.N) {
        case 1: k_op_build<1><<<grid, 256, 0, s>>>(k, b, rk, force ? 1 : 0); break;
        case 2: k_op_build<2><<<grid, 256, 0, s>>>(k, b, rk, force ? 1 : 0); break;
        case 3: k_op_build<3><<<grid, 256, 0, s>>>(k, b, rk, force ? 1 : 0); break;
        case 4: k_op_build<4><<<grid, 256, 0, s>>>(k, b, rk, force ? 1 : 0); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

namespace {
int g_op_resident[5] = {0, 0, 0, 0, 0};   // blocks of k_op_apply<N> resident on the device at once
}

cudaError_t prepare_op_apply() {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* fns[4] = {(const void*)k_op_apply<1>, (const void*)k_op_apply<2>, (const void*)k_op_apply<3>,
                          (const void*)k_op_apply<4>};
    const size_t smem[4] = {op_smem_bytes<1>(), op_smem_bytes<2>(), op_smem_bytes<3>(), op_smem_bytes<4>()};
    for (int j = 0; j < 4 && e == cudaSuccess; ++j) {
        int per = 0;
        e = cudaFuncSetAttribute(fns[j], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem[j]);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fns[j], 288, smem[j]);
        g_op_resident[j + 1] = std::max(1, sms * per);
    }
    return e;
}

cudaError_t launch_op_apply(const Consts<float>& k, const Bufs<float>& b, cudaStream_t s) {
    if (!b.op) return cudaErrorInvalidValue;
    if (k.N < 1 || k.N > 4 || g_op_resident[k.N] == 0) return cudaErrorInvalidValue;
    const long long rows = k.row1 - k.row0;
    if (rows <= 0) return cudaSuccess;
    // one row per block at a time; the grid is what the device holds at once
    const unsigned grid = (unsigned)std::min<long long>(rows, g_op_resident[k.N]);
    k_op_src<<<(unsigned)((k.n_pad + 255) / 256), 256, 0, s>>>(k, b);
    switch (k.N) {
        case 1: k_op_apply<1><<<grid, 288, op_smem_bytes<1>(), s>>>(k, b); break;
        case 2: k_op_apply<2><<<grid, 288, op_smem_bytes<2>(), s>>>(k, b); break;
        case 3: k_op_apply<3><<<grid, 288, op_smem_bytes<3>(), s>>>(k, b); break;
        default: k_op_apply<4><<<grid, 288, op_smem_bytes<4>(), s>>>(k, b); break;
    }
    return cudaGetLastError();
}

// Largest live source log-weight (the screen's lmax), one block.
__global__ void __launch_bounds__(1024) k_live_lmax(Consts<float> k, Bufs<float> b) {
    __shared__ float red[32];
    float m = -INFINITY;
    for (long long i = threadIdx.x; i < k.n; i += blockDim.x)
        if (!b.mask[i]) m = fmaxf(m, b.logw[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
        b.stats->scr_lmax = m;
    }
}

// Screened float32 form: first pass over k1 coordinates (a multiple of 64, 64 <= k1 <= r
// rounded up to 64: the first-pass norms come in chunks of 64), then exact evaluation of
// every tile that keeps a candidate.
cudaError_t launch_ksum_scr32(const Consts<float>& k, const Bufs<float>& b, int k1, cudaStream_t s) {
    if (!b.nu_chunk) return cudaErrorInvalidValue;
    const int rk = ((k.r + BK - 1) / BK) * BK;
    k1 = ((k1 + 63) / 64) * 64;
    if (k1 < 64) k1 = 64;
    if (k1 > k.r_pad) k1 = k.r_pad;
    const unsigned grid = (unsigned)((k.row1 - k.row0 + BM - 1) / BM);   // the handle's target blocks
    if (grid == 0) return cudaSuccess;
    k_live_lmax<<<1, 1024, 0, s>>>(k, b);
    switch (k.N) {
        case 1: k_ksum_scr32<1><<<grid, 256, 0, s>>>(k, b, rk, k1); break;
        case 2: k_ksum_scr32<2><<<grid, 256, 0, s>>>(k, b, rk, k1); break;
        case 3: k_ksum_scr32<3><<<grid, 256, 0, s>>>(k, b, rk, k1); break;
        case 4: k_ksum_scr32<4><<<grid, 256, 0, s>>>(k, b, rk, k1); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// batched: trajectory = blockIdx.y; blocks past a trajectory's rows return at once
template <typename T, int N>
__global__ void __launch_bounds__(256) kb_ksum_simt(const Traj<T>* __restrict__ tr) {
    const Traj<T>& t = tr[blockIdx.y];
    if (t.path == 0 || (long long)blockIdx.x * BM >= t.k.n_pad) return;
    const int rk = ((t.k.r + BK - 1) / BK) * BK;
    ksum_simt_body<T, N>(t.k, t.b, rk, blockIdx.x);
}

template <typename T>
cudaError_t launch_ksum_simt_batch(const Traj<T>* d_traj, int B, int N, long long n_pad_max, int r_max,
                                   cudaStream_t s, int* launches) {
    (void)r_max;
    const dim3 grid((unsigned)(n_pad_max / BM), B);
    switch (N) {
        case 1: kb_ksum_simt<T, 1><<<grid, 256, 0, s>>>(d_traj); break;
        case 2: kb_ksum_simt<T, 2><<<grid, 256, 0, s>>>(d_traj); break;
        case 3: kb_ksum_simt<T, 3><<<grid, 256, 0, s>>>(d_traj); break;
        case 4: kb_ksum_simt<T, 4><<<grid, 256, 0, s>>>(d_traj); break;
        default: return cudaErrorInvalidValue;
    }
    if (launches) *launches += 1;
    return cudaGetLastError();
}
template cudaError_t launch_ksum_simt_batch<float>(const Traj<float>*, int, int, long long, int, cudaStream_t, int*);
template cudaError_t launch_ksum_simt_batch<double>(const Traj<double>*, int, int, long long, int, cudaStream_t, int*);

// Source ranges per target block of the plain form: enough blocks for two per SM (at most
// kSimtMaxSplit ranges, none beyond the source tiles), when the filter has few target
// blocks and the workspace holds the partial states.
int simt_splits(long long n_pad, long long tiles, bool has_part) {
    if (!has_part || tiles <= 0) return 1;
    long long sp = (2 * 152 + tiles - 1) / tiles;
    sp = std::min<long long>(sp, kSimtMaxSplit);
    sp = std::min<long long>(sp, n_pad / BN);
    return (int)std::max<long long>(sp, 1);
}

template <typename T>
cudaError_t launch_ksum_simt(const Consts<T>& k, const Bufs<T>& b, cudaStream_t s, int* launches) {
    const int rk = ((k.r + BK - 1) / BK) * BK;
    const long long tiles = (k.row1 - k.row0 + BM - 1) / BM;   // the handle's target blocks
    if (tiles == 0) return cudaSuccess;
    const int nsplit = simt_splits(k.n_pad, tiles, b.simt_part != nullptr);
    const unsigned grid = (unsigned)(tiles * nsplit);
    const bool noise = (k.noise == YY_NOISE_DIAG);
#define YY_SIMT(NN)                                                                                     \
    case NN:                                                                                            \
        if (noise) k_ksum_simt<T, NN, true><<<grid, 256, 0, s>>>(k, b, rk, nsplit);                     \
        else k_ksum_simt<T, NN><<<grid, 256, 0, s>>>(k, b, rk, nsplit);                                \
        if (nsplit > 1) {                                                                               \
            const unsigned mg = (unsigned)((k.row1 - k.row0 + 255) / 256);                              \
            if (noise) k_simt_merge<T, NN, true><<<mg, 256, 0, s>>>(k, b, nsplit);                      \
            else k_simt_merge<T, NN><<<mg, 256, 0, s>>>(k, b, nsplit);                                 \
        }                                                                                               \
        break;
    switch (k.N) {
        YY_SIMT(1)
        YY_SIMT(2)
        YY_SIMT(3)
        YY_SIMT(4)
        default: return cudaErrorInvalidValue;
    }
#undef YY_SIMT
    if (launches) *launches += (nsplit > 1) ? 2 : 1;
    return cudaGetLastError();
}
template cudaError_t launch_ksum_simt<float>(const Consts<float>&, const Bufs<float>&, cudaStream_t, int*);
template cudaError_t launch_ksum_simt<double>(const Consts<double>&, const Bufs<double>&, cudaStream_t, int*);

}  // namespace yy
