// Prediction step on the 5th-generation tensor cores (sm_103a): Gram screening on tcgen05
// (BF16 or e4m3 operands) + exact float32 evaluation of the surviving pairs.
//
// The kernel sum of the prediction ("Solving Kolmogorov Equations via Low-Discrepancy Sampling
// and Kernel Approximation", eq. general_kernel; "Log-Domain Computation") is, per
// target i and scale j, a log-sum-exp over sources s of
//     score_j(i, s) = -|u_i - tau_j f_i - u_s|^2 / (2 tau_j) + ell_s.
// In high dimension almost every term is smaller than the largest one by hundreds of
// nats, so it is computed as a flash-attention-style tile loop that never materialises the
// n x n matrix and only spends exponentials where they matter:
//
//  1. G = U_t U_s^T on tcgen05 (BF16 operands, or e4m3 copies of s u, staged by TMA in
//     128-byte-swizzled shared memory, FP32 accumulators in TMEM, double-buffered so the
//     MMA of source tile t+1 overlaps the screening of tile t), first over a prefix of the
//     coordinates (a lower bound of the distance), the tiles that keep candidates again
//     over all of them;
//  2. |u_i - u_s|^2 ~= |u_i|^2 + |u_s|^2 - 2 G with a rigorous error bound
//     (|dG| <= 2^-6 |u_i||u_s| for BF16 operands with FP32 accumulation; for e4m3
//     0.14 |u_i||u_s| + 1.07 delta sqrt(K) (|u_i| + |u_s|) + K delta^2, delta = 2^-10 / s;
//     plus float32 rounding), tested per 32 columns first through the largest accumulator
//     and the smallest |u_s|^2, then per column;
//  3. by the triangle inequality |u_i - tau f_i - u_s| >= |u_i - u_s| - tau |f_i|, a pair
//     whose distance exceeds rho_i = max_j [tau_j |f_i| + sqrt(2 tau_j max(0, lmax - M_j(i)
//     + T))] has score_j < M_j(i) - T for every scale, where M_j(i) is the running maximum
//     of exact scores (a lower bound of the row maximum; it starts at the exact self term)
//     and lmax the largest source log-weight of the tile.  With T = ln n + 20 the skipped
//     terms add at most e^-20 relative mass;
//  4. pairs that survive the screen are evaluated exactly in float32 from the float32
//     node coordinates (difference form; for r > 64 warp-cooperative over the
//     coordinates, one pair at a time; for r <= 64 each lane evaluates its own row's
//     pairs) and fed to the online log-sum-exp of their target row.
//
// The screen pays off when few pairs survive (high r: at r >= 100 essentially only the
// self terms).  At low r most pairs are within reach of the kernel and the plain FP32
// form is faster; the batch autotuner routes such filters there.
//
// Work item = one tile of 128 targets of one filter over one of nsplit contiguous ranges
// of that filter's source tiles (BN = 256 or 128 sources per tile).  Every launch is a
// persistent grid in which each CTA walks its own list of items, prepared on the host by
// a longest-processing-time-first assignment; splitting the sources of a target tile
// fills the last wave (a filter with 512 target tiles on 152 SMs would otherwise leave
// 16 % of the SMs idle).  An item over part of the sources stores its rows' online
// (max, sum) states and a merge kernel combines them.  For a batch the TMA descriptors of
// every filter live in global memory.  Warp roles:
// warp 0 issues TMA loads (a tile's coordinate chunks as soon as ring slots free up, its
// q values once the epilogue has released the tile's accumulator), warp 1 allocates TMEM
// and issues tcgen05.mma (one thread), warps 2-9 read the accumulators with tcgen05.ld
// (two warps per TMEM lane quarter, each on half of a tile's columns, one target row per
// thread) and screen.  Every wait is bounded (%globaltimer); on expiry the
// kernel records YY_ERR_TIMEOUT in the status word, drains its own copies and MMAs with a
// bounded wait, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "yy_combine.cuh"
#include "yy_drift.cuh"
#include "yy_tcgen05.cuh"

namespace yy {

namespace tc {
constexpr int BM = 128;      // targets per item (UMMA M)
constexpr int BK = 64;       // coordinates per stage: 64 bf16 = one 128-byte swizzle row
constexpr int UK = 16;       // K of one tcgen05.mma kind::f16
constexpr int EPI_WARPS = 8;  // two per TMEM lane quarter, each on half of a tile's columns
constexpr int NUM_THREADS = 64 + 32 * EPI_WARPS;
constexpr int A_BYTES = BM * BK * 2;
constexpr unsigned long long kTimeoutNs = 4000000000ull;   // default wait limit; drain limit
constexpr float kDeadQ = 3.0e38f;
constexpr float kThetaMax = 1.0e30f;
constexpr int kEscWords = 32;    // per epilogue warp and parity: marks of up to 1024 source tiles
constexpr int kEscThresh = 8;    // candidates of one warp in one tile above which it is rescreened
constexpr int kExactBudget = 64; // exact pairs one warp evaluates per item in the first pass

// Shape-dependent constants.  BN = 256: 4 stages, 512 TMEM columns, one CTA per SM.
// BN = 128: 3 stages (96 KB), 256 TMEM columns, so two CTAs fit on one SM.  PAIR (BN = 256
// only): the two CTAs of a cluster share each source tile, each staging half of it (128
// rows) next to its own 128 target rows, so a stage is 32 KB and the same shared memory
// holds 6 of them; the expected bytes of a stage on the even CTA's barrier cover both.
template <int BN, bool PAIR = false>
struct Cfg {
    static constexpr int STAGES = PAIR ? 6 : ((BN == 256) ? 4 : 3);
    static constexpr int B_BYTES = (PAIR ? BN / 2 : BN) * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t TX_BYTES = (PAIR ? 2u : 1u) * (uint32_t)STAGE_BYTES;
    static constexpr int MMA_M = PAIR ? 2 * BM : BM;
    // buffers of the per-tile source values (q, column bounds, chunk maxima): a ring of its
    // own, so that a tile's values are staged well before its accumulator is ready
    static constexpr int QB = (BN == 256) ? 4 : 2;
    static constexpr uint32_t TMEM_COLS = 2 * BN;   // two accumulators of BN fp32 columns
    static constexpr int HALF = BN / 2;   // columns of one epilogue warp
    // ring | row- and column-direction q values per accumulator | candidate masks per
    // epilogue warp | marking bitmaps | row states exchanged between the two warps of a lane
    // quarter | barriers
    static constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 2 * QB * BN * 4 + QB * 16 * 4 +
                                      2 * EPI_WARPS * HALF * 4 + EPI_WARPS * 2 * kEscWords * 4 +
                                      128 * kMaxScales * 2 * 4 + QB * (BN / 32) * 4 + 384;
    // kind::f16 instruction descriptor: D fp32 (bits 4-5 = 1), A bf16 (bits 7-9 = 1),
    // B bf16 (bits 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                      ((uint32_t)(MMA_M >> 4) << 24);
    // kind::f8f6f4 instruction descriptor: D fp32 (bits 4-5 = 1), A and B e4m3 (bits 7-9 and
    // 10-12 = 0), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
    static constexpr uint32_t IDESC8 = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(MMA_M >> 4) << 24);
};

}  // namespace tc

namespace {

using namespace ptx;

// Bounded wait: false when the limit expired (status recorded) or another role aborted.
// CL: acquire at cluster scope (waits after which the other CTA of a pair's shared memory
// is read).
template <bool CL = false>
__device__ __forceinline__ bool try_wait_sc(uint64_t* bar, uint32_t parity) {
    return CL ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity);
}
template <bool CL = false>
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                             unsigned int* status, unsigned long long limit_ns) {
    if (try_wait_sc<CL>(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (try_wait_sc<CL>(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > limit_ns) {
            *abort_flag = 1;
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
}
// Untiled bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
// completing on an mbarrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    uint64_t g;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(reinterpret_cast<uint64_t>(src)));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(g), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Bounded wait used while draining after an abort (ignores the abort flag).
__device__ __forceinline__ void wait_drain(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > tc::kTimeoutNs) return;
}
// the largest of three floats (exact)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// the smallest of three floats (exact)
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
// An upper bound of sqrt(x) for x >= 0: x times the reciprocal square root (hardware
// approximation, relative error far below 1e-6), widened by 1e-6.  The screen only needs
// its radii not to be underestimated.
__device__ __forceinline__ float sqrt_up(float x) {
    return x > 0.f ? x * rsqrtf(x) * 1.000001f : 0.f;
}

// Screening threshold on |u_s|^2 - 2 G for one target row (see the file comment).  rnu_i
// and rnumax are the square roots of nu_i and numax (per row and per tile, precomputed).
template <int N>
__device__ __forceinline__ float screen_theta(const Consts<float>& k, bool live, float nu_i, float rnu_i, float Fi,
                                              const float (&mx)[N], float lmax, float numax, float rnumax,
                                              float T) {
    if (!live || lmax == -INFINITY) return -INFINITY;
    float rho = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (mx[j] == -INFINITY) return tc::kThetaMax;
        const float gap = fmaxf(lmax - mx[j] + T, 0.f);
        rho = fmaxf(rho, k.tau[j] * Fi + sqrt_up(2.f * k.tau[j] * gap));
    }
    const float err = 2.f * k.tc_eps * rnu_i * rnumax + k.tc_dabs * (rnu_i + rnumax) + k.tc_dabs2 +
                      2e-6f * (nu_i + numax + rho * rho);
    return fminf(rho * rho + err - nu_i, tc::kThetaMax);
}

}  // namespace

// Coordinate stages of one filter's screen: 64 coordinates (BF16) or 128 (FP8, rows of
// tc_r8 bytes) per stage.
__device__ __forceinline__ int screen_stages(const Consts<float>& k) {
    return k.tc_fp8 ? k.tc_r8 / 128 : k.r_pad / tc::BK;
}
// Chunks of 64 coordinates covered by the first `stages` stages (for the restricted norms).
__device__ __forceinline__ int stage_chunks64(const Consts<float>& k, int stages) {
    return k.tc_fp8 ? min(2 * stages, k.r_pad / 64) : stages;
}

// First-pass stages of one filter's screen: fixed by the configuration, else the
// controller's last choice (tc_adapt), else half of the stages (the controller finds the
// shortest clean length from above).
__device__ __forceinline__ int prefix_chunks(const Consts<float>& k, const DevStats* st) {
    const int nk = screen_stages(k);
    int v = k.tc_prefix > 0 ? k.tc_prefix : st->tc_nk1;
    if (v <= 0) v = (nk + 1) / 2;
    return v < 1 ? 1 : (v > nk ? nk : v);
}

// Drift component d of node row `row` at x = c + u: the stored f where the preparation pass
// writes it, else recomputed with that pass's arithmetic (per-dimension constants dimc),
// which gives the value it would have stored.
__device__ __forceinline__ float drift_at(const Consts<float>& k, const Bufs<float>& b, long long row, float u, int d) {
    const int rp = k.r_pad;
    if (b.store_f) return b.f[(size_t)row * rp + d];
    if (k.model == YY_MODEL_CUBIC) {
        float fv, sn;
        cubic_drift(u, b.dimc[d], b.dimc[rp + d], b.dimc[3 * rp + d], b.dimc[4 * rp + d], &fv, &sn);
        return fv;
    }
    return k.model_a * (b.dimc[d] + (u + b.dimc[rp + d]));
}

// Exact pair sums of target row tgt and source row src, warp-cooperative over the
// coordinates: s1 = |u_t - u_s|^2 and s2 = (u_t - u_s) . f(x_t), each lane over the
// coordinates lane, lane + 32, ... in increasing order (then summed across the warp by the
// caller).  Four coordinates per lane are loaded before any is used, so that a pair costs
// r / 128 memory round trips rather than r / 32.
__device__ __forceinline__ void pair_sums_warp(const Consts<float>& k, const Bufs<float>& b, long long tgt,
                                               long long src, int lane, float& s1, float& s2) {
    const float* ut = b.u + (size_t)tgt * k.r_pad;
    const float* us = b.u + (size_t)src * k.r_pad;
    const float* ft = b.f + (size_t)tgt * k.r_pad;
    const bool sf = b.store_f != 0;
    s1 = 0.f;
    s2 = 0.f;
    for (int d0 = 0; d0 < k.r; d0 += 128) {
        float a[4], c[4], g[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int d = d0 + 32 * m + lane;
            const bool in = d < k.r;
            a[m] = in ? ut[d] : 0.f;
            c[m] = in ? us[d] : 0.f;
            g[m] = (in && sf) ? ft[d] : 0.f;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int d = d0 + 32 * m + lane;
            if (d < k.r) {
                const float dl = a[m] - c[m];
                s1 = fmaf(dl, dl, s1);
                s2 = fmaf(dl, sf ? g[m] : drift_at(k, b, tgt, a[m], d), s2);
            }
        }
    }
}

// Per source chunk of 128: |u_s|^2 of live sources over all coordinates (tc_q) and over the
// first-pass coordinates (tc_q1), kDeadQ for masked, padded or -inf ones; the largest live
// log-weight; the largest live value of each kind of |u_s|^2.
__device__ __forceinline__ void colprep_body(const Consts<float>& k, const Bufs<float>& b, int chunk) {
    __shared__ float red_l[4], red_n[4], red_n1[4];
    const long long s = (long long)chunk * 128 + threadIdx.x;
    const int nkc = k.r_pad / 64;
    const int nk1 = stage_chunks64(k, prefix_chunks(k, b.stats));
    float lw = -INFINITY, nu = 0.f, nu1 = 0.f;
    bool live = false;
    if (s < k.n) {
        lw = b.logw[s];
        nu = b.nu[s];
        const float* nc = b.nu_chunk + (size_t)s * nkc;
        for (int c = 0; c < nk1; ++c) nu1 += nc[c];
        live = !b.mask[s] && lw != -INFINITY;
    }
    b.tc_q[s] = live ? nu : tc::kDeadQ;
    b.tc_q1[s] = live ? nu1 : tc::kDeadQ;
    b.tc_q1t[s] = nu1;
    {   // the smallest of each group of 32 (one warp), for the screen's first test
        float qa = live ? nu : tc::kDeadQ, qb = live ? nu1 : tc::kDeadQ;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            qa = fminf(qa, __shfl_xor_sync(0xffffffffu, qa, o));
            qb = fminf(qb, __shfl_xor_sync(0xffffffffu, qb, o));
        }
        if ((threadIdx.x & 31) == 0) {
            b.tc_qmin[s >> 5] = qa;
            b.tc_qmin1[s >> 5] = qb;
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxScales; ++j) b.tc_xlse[(size_t)s * kMaxScales + j] = 0ull;   // empty (sum 0)
    float lm = live ? lw : -INFINITY, nm = live ? nu : 0.f, nm1 = live ? nu1 : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lm = fmaxf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
        nm = fmaxf(nm, __shfl_xor_sync(0xffffffffu, nm, o));
        nm1 = fmaxf(nm1, __shfl_xor_sync(0xffffffffu, nm1, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red_l[threadIdx.x >> 5] = lm;
        red_n[threadIdx.x >> 5] = nm;
        red_n1[threadIdx.x >> 5] = nm1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 4; ++w) {
            lm = fmaxf(lm, red_l[w]);
            nm = fmaxf(nm, red_n[w]);
            nm1 = fmaxf(nm1, red_n1[w]);
        }
        b.tc_tile_lmax[chunk] = lm;
        b.tc_tile_numax[chunk] = nm;
        b.tc_tile_numax1[chunk] = nm1;
        float* ci = b.tc_cinfo + (size_t)chunk * 8;   // staged per tile by the prediction's producer
        ci[0] = lm;
        ci[1] = nm;
        ci[2] = nm1;
        ci[5] = sqrt_up(nm);    // square roots of the norm maxima, for the screen's error term
        ci[6] = sqrt_up(nm1);
        ci[7] = 0.f;
    }
}

__global__ void __launch_bounds__(128) k_tc_colprep(Consts<float> k, Bufs<float> b) { colprep_body(k, b, blockIdx.x); }

__global__ void __launch_bounds__(128) kb_tc_colprep(const Traj<float>* __restrict__ tr) {
    const Traj<float>& t = tr[blockIdx.y];
    if (t.path != 0 || (long long)blockIdx.x * 128 >= t.k.n_pad) return;
    colprep_body(t.k, t.b, blockIdx.x);
}

// Controller of the first-pass length, run once per prediction launch and filter (by the
// last CTA to finish).  The work beyond the first pass, in chunks per tile, is
//     extra = (rescreened tiles x all chunks + exact pair evaluations x r / 4096) / tiles
// (an exact pair costs about r / 4096 of the tensor time of one chunk of one tile).  A
// length is acceptable when extra <= 1/50 and clean when extra = 0.  After an unacceptable
// prediction the length grows at once (by 2 when extra > 4) and the one just used is held
// off for 1024 predictions; after four clean predictions in a row at one length, one chunk
// shorter is tried unless it is held off.  A shorter length that is acceptable but not
// clean is given up at once for the clean one it came from (and held off): every exact
// pair stalls its epilogue warp for the memory latency of a whole row, so a few hundred
// of them cost more than the chunk they save (measured at r = 1000, n = 65536, FP8: 3 of 8
// stages with 395 exact pairs 1.09 ms, 4 stages and none 0.89 ms).  An acceptable length
// that is not clean and was not reached by shortening is kept.
__device__ void tc_adapt(const Consts<float>& k, DevStats* st) {
    const unsigned long long blk = atomicExch(&st->tc_blk, 0ull);
    const unsigned long long esc = atomicExch(&st->tc_esc, 0ull);
    const unsigned long long cand = atomicAdd(&st->candidates, 0ull);
    const int nk1 = prefix_chunks(k, st);
    st->tc_last_blk = blk;
    st->tc_last_esc = esc;
    st->tc_last_nk1 = nk1;
    if (k.tc_prefix > 0 || blk == 0) return;
    const int nk = screen_stages(k);
    constexpr int kHold = 1024, kSettle = 4;
    for (int x = 1; x <= nk; ++x)
        if (st->tc_hold[x] > 0) --st->tc_hold[x];
    const int from = st->tc_from;
    st->tc_from = nk1;
    const double extra = ((double)esc * nk + (double)cand * k.r / 4096.0) / (double)blk;
    int next = nk1;
    if (extra > 0.02) {
        st->tc_streak = 0;
        if (nk1 < nk) {
            st->tc_hold[nk1] = kHold;
            next = min(nk, nk1 + (extra > 4.0 ? 2 : 1));
        }
    } else {
        const bool clean = esc == 0 && cand == 0;
        if (!clean && from > nk1) {
            // a shortening step that is not clean: return to the clean length it came from
            st->tc_hold[nk1] = kHold;
            next = from;
            st->tc_streak = 0;
        } else {
            st->tc_streak = clean ? ((from == nk1) ? st->tc_streak + 1 : 1) : 0;
            if (st->tc_streak >= kSettle && nk1 > 1 && st->tc_hold[nk1 - 1] == 0) {
                next = nk1 - 1;
                st->tc_streak = 0;
            }
        }
    }
    st->tc_nk1 = next;
}

// Column direction of the symmetric screen, per node c as a target: every source s with
// |u_c - u_s| <= rho_c can carry more than e^-T of c's row, where, as in the row direction,
//     rho_c = max_j [tau_j |f_c| + sqrt(2 tau_j max(0, lmax - M_j(c) + T))],
// but with the reference M_j(c) = the exact self term of c (a lower bound of the row
// maximum) and lmax the largest live log-weight of all sources.  The screen compares
// |u_i|^2 + |u_c|^2 - 2 G with rho_c^2 + err_c (err_c as in the row direction, with the
// largest live |u_s|^2); stored is |u_c|^2 - (rho_c^2 + err_c), over all coordinates (tc_qt)
// and over the first-pass coordinates (tc_qt1).  Masked or padded nodes are no targets
// (+inf); a live node without a finite log-weight has no reference (-inf: every pair).
__device__ __forceinline__ void colprep2_body(const Consts<float>& k, const Bufs<float>& b, int chunk) {
    __shared__ float red[3][4];
    const int nch = (int)(k.n_pad / 128);
    float lg = -INFINITY, ng = 0.f, ng1 = 0.f;
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
        lg = fmaxf(lg, b.tc_tile_lmax[c]);
        ng = fmaxf(ng, b.tc_tile_numax[c]);
        ng1 = fmaxf(ng1, b.tc_tile_numax1[c]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lg = fmaxf(lg, __shfl_xor_sync(0xffffffffu, lg, o));
        ng = fmaxf(ng, __shfl_xor_sync(0xffffffffu, ng, o));
        ng1 = fmaxf(ng1, __shfl_xor_sync(0xffffffffu, ng1, o));
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = lg; red[1][threadIdx.x >> 5] = ng; red[2][threadIdx.x >> 5] = ng1; }
    __syncthreads();
    for (int w = 0; w < 4; ++w) { lg = fmaxf(lg, red[0][w]); ng = fmaxf(ng, red[1][w]); ng1 = fmaxf(ng1, red[2][w]); }
    const long long c = (long long)chunk * 128 + threadIdx.x;
    float qt = INFINITY, qt1 = INFINITY;
    if (c < k.n && !b.mask[c] && lg != -INFINITY) {
        const float lc = b.logw[c];
        if (lc == -INFINITY) {
            qt = qt1 = -INFINITY;
        } else {
            const float T = logf((float)k.n) + 20.0f;
            const float nfc = b.nf[c], Fc = sqrtf(nfc);
            float rho = 0.f;
#pragma unroll 4
            for (int j = 0; j < k.N; ++j) {
                const float gap = fmaxf(lg - (-0.5f * k.tau[j] * nfc + lc) + T, 0.f);
                rho = fmaxf(rho, k.tau[j] * Fc + sqrtf(2.f * k.tau[j] * gap));
            }
            const float q = b.nu[c], q1 = b.tc_q1t[c];
            const float e = 2.f * k.tc_eps * sqrtf(q * ng) + k.tc_dabs * (sqrtf(q) + sqrtf(ng)) + k.tc_dabs2 +
                            1e-6f * (q + ng + rho * rho);
            const float e1 = 2.f * k.tc_eps * sqrtf(q1 * ng1) + k.tc_dabs * (sqrtf(q1) + sqrtf(ng1)) + k.tc_dabs2 +
                             1e-6f * (q1 + ng1 + rho * rho);
            qt = q - fminf(rho * rho + e, tc::kThetaMax);
            qt1 = q1 - fminf(rho * rho + e1, tc::kThetaMax);
        }
    }
    b.tc_qt[c] = qt;
    b.tc_qt1[c] = qt1;
    // the chunk's largest bound rho_c^2 + err_c (targets only; -inf value: unbounded)
    __shared__ float rr[2][4];
    float r0 = (qt == INFINITY) ? 0.f : (qt == -INFINITY ? INFINITY : b.nu[c] - qt);
    float r1 = (qt1 == INFINITY) ? 0.f : (qt1 == -INFINITY ? INFINITY : b.tc_q1t[c] - qt1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        r0 = fmaxf(r0, __shfl_xor_sync(0xffffffffu, r0, o));
        r1 = fmaxf(r1, __shfl_xor_sync(0xffffffffu, r1, o));
    }
    if ((threadIdx.x & 31) == 0) { rr[0][threadIdx.x >> 5] = r0; rr[1][threadIdx.x >> 5] = r1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 4; ++w) { r0 = fmaxf(r0, rr[0][w]); r1 = fmaxf(r1, rr[1][w]); }
        // widened by float rounding of q_c - (q_c - R_c), so the combined test stays conservative
        b.tc_tile_rmax[chunk] = r0 + 1e-6f * (fabsf(r0) + 1.f);
        b.tc_tile_rmax1[chunk] = r1 + 1e-6f * (fabsf(r1) + 1.f);
        b.tc_cinfo[(size_t)chunk * 8 + 3] = b.tc_tile_rmax[chunk];
        b.tc_cinfo[(size_t)chunk * 8 + 4] = b.tc_tile_rmax1[chunk];
    }
}

__global__ void __launch_bounds__(128) k_tc_colprep2(Consts<float> k, Bufs<float> b) { colprep2_body(k, b, blockIdx.x); }

// Adds e^score to a log-sum-exp accumulator kept as one 64-bit word (low half: running
// maximum, high half: sum of e^(term - maximum); sum 0 = empty) by compare-and-swap.  Every
// failed exchange means another thread's update went through, so the loop ends; it is
// capped all the same, with the status word recording a give-up.
__device__ __forceinline__ void lse_atomic_add(unsigned long long* w, float score, unsigned int* status) {
    unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(w);
    for (int tries = 0; tries < (1 << 20); ++tries) {
        const float m = __uint_as_float((uint32_t)old), sm = __uint_as_float((uint32_t)(old >> 32));
        float m2, s2;
        if (sm == 0.f) { m2 = score; s2 = 1.f; }
        else if (score > m) { m2 = score; s2 = fmaf(sm, expf(m - score), 1.f); }
        else { m2 = m; s2 = sm + expf(score - m); }
        const unsigned long long nw = (unsigned long long)__float_as_uint(m2) |
                                      ((unsigned long long)__float_as_uint(s2) << 32);
        const unsigned long long seen = atomicCAS(w, old, nw);
        if (seen == old) return;
        old = seen;
    }
    atomicOr(status, kStatusTimeout);
}

// Work list of a launch: CTA c processes items[cta_start[c] .. cta_start[c + 1]), each
// (filter, target tile, split, nsplit): target rows 128 tile .. +127 against source tiles
// [nst split / nsplit, nst (split + 1) / nsplit).  tr == nullptr: single filter, passed by
// value with its TMA maps; otherwise descriptors tr[filter] (nb filters) and TMA maps
// maps[2 filter] (A, 128-row box) and maps[2 filter + 1] (B, BN-row box).
struct TcWork {
    const Traj<float>* tr;
    const CUtensorMap* maps;
    const int4* items;
    const int* cta_start;
    int nb;
    unsigned long long wait_ns;   // limit of every bounded wait (the drain after an abort keeps 4 s)
};

constexpr int kMaxSplit = 8;

// Partial online log-sum-exp states of split items: [row][split][scale] (max, sum).
__device__ __forceinline__ float* part_slot(const Bufs<float>& b, long long i, int split, int j) {
    return b.tc_part + (((size_t)i * kMaxSplit + split) * kMaxScales + j) * 2;
}

// Two-pass screen of one item.  Pass 1 runs the Gram product over the first nk1 of nk
// coordinate chunks only: restricted to them, |u_i - u_s| is still a lower bound of the full
// distance, so the same test (with the restricted norms) rejects pairs rigorously.  An
// epilogue warp whose 32 rows keep more than kEscThresh candidates in a tile marks the tile
// for pass 2 instead of evaluating them; after pass 1 of the item the three roles meet at
// an mbarrier, and pass 2 recomputes the marked tiles over all coordinates and screens them
// again (only the marking warps use the result).  With nk1 = nk there is one pass.
//
// PAIR: the grid is made of 2-CTA clusters (one CTA per SM) and work item p of a cluster
// is the pair of target tiles 2p (even CTA) and 2p + 1 (odd CTA), which have the same
// source range.  Each CTA stages its own 128 target rows and half of each source tile;
// the even CTA's MMA thread issues tcgen05.mma.cta_group::2 (M = 256) once both halves
// have landed on its barrier, and its commits arrive on the barriers of both CTAs.  The
// even CTA's MMA waits until the epilogues of both CTAs have released an accumulator
// (the odd CTA's arrive remotely).  Tiles to be screened again are the union of both
// CTAs' marks.  Everything else -- screening, exact evaluation, row states -- is per CTA
// and identical to the single-CTA kernel.
template <int N, int BN, bool PAIR>
// One CTA per SM; with 10 warps two of the four SM sub-partitions hold three warps each, so
// the register budget is 168 per thread.
__global__ void __launch_bounds__(tc::NUM_THREADS, 1)
    k_ksum_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ Consts<float> k0, const __grid_constant__ Bufs<float> b0, TcWork w) {
    using namespace tc;
    using C = Cfg<BN, PAIR>;
    static_assert(!PAIR || BN == 256, "CTA pairs share 256-wide source tiles");
    // the waits after which a CTA reads the other CTA's marks acquire at cluster scope; the
    // pipeline waits (ring, accumulators, q buffers) order only asynchronous copies and
    // tensor-core work and stay at CTA scope
    constexpr bool CL = PAIR;
    constexpr int STAGES = C::STAGES;
    constexpr int STAGE_BYTES = C::STAGE_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int HALF = C::HALF;
    // q_s of the tile's sources and, for symmetric blocks, the column-direction values,
    // staged by the producer per accumulator: [2][BN] each
    constexpr int QB = C::QB;
    float* qbuf = reinterpret_cast<float*>(smem + STAGES * STAGE_BYTES);   // [QB][BN]
    float* qtbuf = qbuf + QB * BN;                                         // [QB][BN]
    float* qinfo = qtbuf + QB * BN;                                        // [QB][16]: the tile's chunk maxima
    float* qmbuf = qinfo + QB * 16;                                        // [QB][BN / 32]: smallest q_s per 32
    uint32_t* cms = reinterpret_cast<uint32_t*>(qmbuf + QB * (BN / 32));   // [EPI_WARPS][HALF / 32][32]
    uint32_t* tcms = cms + EPI_WARPS * HALF;                             // [EPI_WARPS][HALF / 32][32]
    uint32_t* escm = tcms + EPI_WARPS * HALF;                            // [EPI_WARPS][2][kEscWords]
    float* xch = reinterpret_cast<float*>(escm + EPI_WARPS * 2 * kEscWords);   // [128 rows][kMaxScales][2]
    uint64_t* bars = reinterpret_cast<uint64_t*>(xch + 128 * kMaxScales * 2);
    uint64_t* full = bars;
    uint64_t* empty = bars + STAGES;
    uint64_t* tfull = bars + 2 * STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint64_t* escb = drain + 1;
    uint64_t* xfull = escb + 1;    // [4]: the second warp of lane quarter q stored its row states
    uint64_t* xfree = xfull + 4;   // [4]: the first warp of lane quarter q has read them
    uint64_t* qfull = xfree + 4;   // [QB]: the source values of a tile landed in q buffer b
    uint64_t* qempty = qfull + QB; // [QB]: the epilogue is done with q buffer b
    // [2] (pairs, even CTA): accumulator a released by the epilogues of both CTAs; the MMA
    // waits on it (single CTAs: on tempty)
    uint64_t* tpair = qempty + QB;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tpair + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool batched = (w.tr != nullptr);
    const uint32_t rank = PAIR ? cluster_ctarank() : 0u;   // 0: even CTA (issues the MMAs)
    const int unit = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;   // work list index
    const int it_begin = w.cta_start[unit];
    const int it_end = w.cta_start[unit + 1];
    // status word for timeouts: the first filter of this CTA (none if the CTA has no work)
    unsigned int* status = (it_end <= it_begin) ? nullptr
                           : batched ? &w.tr[w.items[it_begin].x].b.stats->status : &b0.stats->status;

    DevStats* const ctr = batched ? w.tr[0].b.stats : b0.stats;   // launch-wide counter
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], EPI_WARPS);
            mbar_init(&tpair[a], 2 * EPI_WARPS);   // both CTAs' epilogue warps
        }
        mbar_init(drain, 1);
        mbar_init(escb, PAIR ? 2 * EPI_WARPS : EPI_WARPS);   // a pair's marks are read by both
        for (int a = 0; a < 4; ++a) { mbar_init(&xfull[a], 1); mbar_init(&xfree[a], 1); }
        for (int a = 0; a < QB; ++a) { mbar_init(&qfull[a], 1); mbar_init(&qempty[a], EPI_WARPS); }
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) {
        if (PAIR) {   // one warp of each CTA; both receive the same column
            tmem_alloc_pair(tmem_slot, C::TMEM_COLS);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(tmem_slot, C::TMEM_COLS);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (PAIR) cluster_sync();   // both CTAs' barriers initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // the other CTA's copies of the barriers and marks a pair uses (shared::cluster)
    const uint32_t full_lead = PAIR ? mapa_shared(full, 0) : 0u;      // the even CTA's ring barriers
    const uint32_t tpair_lead = PAIR ? mapa_shared(tpair, 0) : 0u;
    const uint32_t escb_peer = PAIR ? mapa_shared(escb, rank ^ 1u) : 0u;
    const uint32_t escm_peer = PAIR ? mapa_shared(escm, rank ^ 1u) : 0u;

    // per-item view: descriptors, maps, first target row, source tile range, split, chunks
    // of all coordinates (nk) and of the first pass (nk1; nk when the range does not fit
    // the marking bitmaps)
    auto item_kb = [&](int idx, const Consts<float>*& kp, const Bufs<float>*& bp, const CUtensorMap*& ma,
                       const CUtensorMap*& mb, long long& i0, int& t0, int& t1, int& split, int& nsplit, int& nk,
                       int& nk1) {
        const int4 it = w.items[idx];
        if (!batched) {
            kp = &k0; bp = &b0; ma = &tmA; mb = &tmB;
        } else {
            kp = &w.tr[it.x].k; bp = &w.tr[it.x].b;
            ma = &w.maps[2 * it.x]; mb = &w.maps[2 * it.x + 1];
        }
        i0 = PAIR ? (long long)it.y * (2 * BM) + (long long)rank * BM : (long long)it.y * BM;
        split = it.z;
        nsplit = it.w;
        // symmetric screen: only source tiles from the one holding the tile's first row on
        const int nst = (int)(kp->n_pad / BN);
        const int bmin = kp->tc_sym ? (int)(i0 / BN) : 0;
        const int L = nst - bmin;
        t0 = bmin + (int)(((long long)L * split) / nsplit);
        t1 = bmin + (int)(((long long)L * (split + 1)) / nsplit);
        nk = screen_stages(*kp);
        nk1 = (t1 - t0 <= kEscWords * 32) ? prefix_chunks(*kp, bp->stats) : nk;
    };
    // tile j of the item marked by epilogue warp e / by any epilogue warp (bitmap parity par)
    auto esc_bit = [&](int e, uint32_t par, int j) -> bool {
        return (escm[(e * 2 + par) * kEscWords + (j >> 5)] >> (j & 31)) & 1u;
    };
    // a pair screens again the union of both CTAs' marks
    auto esc_any = [&](uint32_t par, int j) -> bool {
        bool m = false;
#pragma unroll
        for (int e = 0; e < EPI_WARPS; ++e) m |= esc_bit(e, par, j);
        if (PAIR && !m) {
#pragma unroll
            for (int e = 0; e < EPI_WARPS; ++e)
                m |= (ld_shared_cluster_u32(escm_peer + (uint32_t)(((e * 2 + (int)par) * kEscWords + (j >> 5)) * 4)) >>
                      (j & 31)) & 1u;
        }
        return m;
    };

    if (warp == 0) {
        if (lane == 0 && status) {
            // ---- TMA producer -------------------------------------------------------
            int last_phase[STAGES];
            for (int s = 0; s < STAGES; ++s) last_phase[s] = -1;
            int last_qphase[QB];
            for (int a = 0; a < QB; ++a) last_qphase[a] = -1;
            uint32_t it = 0, npre = 0, tp = 0;
            bool ok = true;
            // one tile: its source values into the next q buffer (free once the epilogue is
            // done with the tile QB back, so they are staged well ahead), then its
            // coordinate chunks into the ring (gated by the ring's slots only, so they
            // stream in while the epilogue still holds the accumulator)
            auto load_tile = [&](const Consts<float>* kp, const Bufs<float>* bp, const CUtensorMap* ma,
                                 const CUtensorMap* mb, long long i0, int t, int nkb, bool prefix) -> bool {
                const int qs = (int)(tp % QB);
                const uint32_t qph = (tp / QB) & 1u;
                ++tp;
                if (!wait_bounded(&qempty[qs], qph ^ 1u, abort_flag, status, w.wait_ns)) return false;
                const uint32_t qb = (uint32_t)(BN * sizeof(float));
                const uint32_t ib = (uint32_t)((BN / 128) * 8 * sizeof(float));
                const uint32_t qmb = (uint32_t)((BN / 32) * sizeof(float));
                mbar_arrive_expect_tx(&qfull[qs], (kp->tc_sym ? 2 * qb : qb) + ib + qmb);
                bulk_load(qbuf + qs * BN, (prefix ? bp->tc_q1 : bp->tc_q) + (size_t)t * BN, qb, &qfull[qs]);
                bulk_load(qinfo + qs * 16, bp->tc_cinfo + (size_t)t * (BN / 128) * 8, ib, &qfull[qs]);
                bulk_load(qmbuf + qs * (BN / 32), (prefix ? bp->tc_qmin1 : bp->tc_qmin) + (size_t)t * (BN / 32), qmb,
                          &qfull[qs]);
                if (kp->tc_sym)
                    bulk_load(qtbuf + qs * BN, (prefix ? bp->tc_qt1 : bp->tc_qt) + (size_t)t * BN, qb, &qfull[qs]);
                last_qphase[qs] = (int)qph;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % STAGES);
                    const uint32_t ph = (it / STAGES) & 1u;
                    if (!wait_bounded(&empty[s], ph ^ 1u, abort_flag, status, w.wait_ns)) return false;
                    uint8_t* dA = smem + s * STAGE_BYTES;
                    const int x = kb * (kp->tc_fp8 ? 128 : BK);   // 128 bytes of coordinates per stage
                    if (PAIR) {
                        // this CTA's 128 target rows and source rows t BN + 128 rank .. +127
                        // (the 128-row map serves both), counted on the even CTA's barrier
                        if (rank == 0) mbar_arrive_expect_tx(&full[s], C::TX_BYTES);
                        const uint32_t fb = full_lead + (uint32_t)(s * 8);
                        tma_load_2d_pair(ma, fb, dA, x, (int)i0);
                        tma_load_2d_pair(ma, fb, dA + A_BYTES, x, t * BN + (int)rank * BM);
                    } else {
                        mbar_arrive_expect_tx(&full[s], C::TX_BYTES);
                        tma_load_2d(ma, &full[s], dA, x, (int)i0);
                        tma_load_2d(mb, &full[s], dA + A_BYTES, x, t * BN);
                    }
                    last_phase[s] = (int)ph;
                }
                return true;
            };
            for (int idx = it_begin; idx < it_end && ok; ++idx) {
                const Consts<float>* kp; const Bufs<float>* bp; const CUtensorMap* ma; const CUtensorMap* mb;
                long long i0;
                int t0, t1, split, nsplit, nk, nk1;
                item_kb(idx, kp, bp, ma, mb, i0, t0, t1, split, nsplit, nk, nk1);
                const bool pre = nk1 < nk;
                for (int t = t0; t < t1 && ok; ++t) ok = load_tile(kp, bp, ma, mb, i0, t, nk1, pre);
                if (ok && pre) {
                    const uint32_t par = npre++ & 1u;
                    if (!wait_bounded<CL>(escb, par, abort_flag, status, w.wait_ns)) { ok = false; break; }
                    for (int t = t0; t < t1 && ok; ++t)
                        if (esc_any(par, t - t0)) ok = load_tile(kp, bp, ma, mb, i0, t, nk, false);
                }
            }
            if (!ok) {   // let our own copies land before shared memory is released
                if (!PAIR) {
                    for (int s = 0; s < STAGES; ++s)
                        if (last_phase[s] >= 0) wait_drain(&full[s], (uint32_t)last_phase[s]);
                } else {
                    // a pair's ring barriers count both CTAs' copies (the odd CTA's cannot be
                    // waited on at all, and the even CTA's barrier may wait for the odd CTA's
                    // half that never comes): give this CTA's own copies time to land (a
                    // copy takes microseconds); both CTAs then leave together
                    const unsigned long long tq = globaltimer();
                    while (globaltimer() - tq < 1000000ull) {}
                }
                for (int a = 0; a < QB; ++a)
                    if (last_qphase[a] >= 0) wait_drain(&qfull[a], (uint32_t)last_qphase[a]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && status && rank == 0) {
            // ---- MMA issuer (the even CTA of a pair issues for both) -------------------
            uint32_t it = 0, tcount = 0, npre = 0;
            bool ok = true;
            // the ring slot / accumulator is free again in every CTA that staged into it
            auto commit_all = [&](uint64_t* bar) {
                if (PAIR) mma_commit_pair_mc(bar, (uint16_t)3);
                else mma_commit(bar);
            };
            auto mma_tile = [&](int nkb, bool fp8) -> bool {
                const int acc = (int)(tcount & 1u);
                const uint32_t aph = (tcount >> 1) & 1u;
                uint64_t* rel = PAIR ? &tpair[acc] : &tempty[acc];
                if (!wait_bounded(rel, aph ^ 1u, abort_flag, status, w.wait_ns)) return false;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc * BN);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = (int)(it % STAGES);
                    const uint32_t ph = (it / STAGES) & 1u;
                    if (!wait_bounded(&full[s], ph, abort_flag, status, w.wait_ns)) return false;
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
                    const uint32_t b0a = a0 + A_BYTES;
                    // four instructions per stage either way: K = 16 bf16 or 32 e4m3, 32 bytes
                    if (fp8) {
#pragma unroll
                        for (int kk = 0; kk < BK / UK; ++kk) {
                            if (PAIR)
                                mma_f8_pair(d_tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0a + kk * 32), C::IDESC8,
                                            (kb | kk) != 0 ? 1u : 0u);
                            else
                                mma_f8(d_tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0a + kk * 32), C::IDESC8,
                                       (kb | kk) != 0 ? 1u : 0u);
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < BK / UK; ++kk) {
                            if (PAIR)
                                mma_bf16_pair(d_tmem, sw128_desc(a0 + kk * UK * 2), sw128_desc(b0a + kk * UK * 2),
                                              C::IDESC, (kb | kk) != 0 ? 1u : 0u);
                            else
                                mma_bf16(d_tmem, sw128_desc(a0 + kk * UK * 2), sw128_desc(b0a + kk * UK * 2),
                                         C::IDESC, (kb | kk) != 0 ? 1u : 0u);
                        }
                    }
                    commit_all(&empty[s]);
                }
                commit_all(&tfull[acc]);
                ++tcount;
                return true;
            };
            for (int idx = it_begin; idx < it_end && ok; ++idx) {
                const Consts<float>* kp; const Bufs<float>* bp; const CUtensorMap* ma; const CUtensorMap* mb;
                long long i0;
                int t0, t1, split, nsplit, nk, nk1;
                item_kb(idx, kp, bp, ma, mb, i0, t0, t1, split, nsplit, nk, nk1);
                for (int t = t0; t < t1 && ok; ++t) ok = mma_tile(nk1, kp->tc_fp8 != 0);
                unsigned long long nesc = 0;
                if (ok && nk1 < nk) {
                    const uint32_t par = npre++ & 1u;
                    if (!wait_bounded<CL>(escb, par, abort_flag, status, w.wait_ns)) { ok = false; break; }
                    for (int t = t0; t < t1 && ok; ++t)
                        if (esc_any(par, t - t0)) { ok = mma_tile(nk, kp->tc_fp8 != 0); ++nesc; }
                }
                if (ok) {   // counted in blocks of 128 targets x BN sources (a pair MMA is two)
                    const unsigned long long per = PAIR ? 2ull : 1ull;
                    atomicAdd(&bp->stats->tc_blk, per * (unsigned long long)(t1 - t0));
                    if (nesc) atomicAdd(&bp->stats->tc_esc, per * nesc);
                }
            }
            // all MMAs issued by this thread have completed once drain fires
            if (PAIR) mma_commit_pair(drain);
            else mma_commit(drain);
            wait_drain(drain, 0);
        }
    } else if (status) {
        // ---- epilogue: screening + exact evaluation --------------------------------------
        // warp pair (q, h): TMEM lane quarter q (its 32 target rows), columns h HALF ..
        // h HALF + HALF - 1 of every tile; each warp keeps its own online log-sum-exp of its
        // rows over its columns, and the pair merges them at the end of an item
        // a wait whose outcome every lane of the warp shares (the lanes go on to aligned
        // TMEM loads and warp barriers together, or all leave); cl: acquire at cluster scope
        auto wait_warp = [&](uint64_t* bar, uint32_t parity, bool cl = false) -> bool {
            const bool got = cl ? wait_bounded<true>(bar, parity, abort_flag, status, w.wait_ns)
                                : wait_bounded<false>(bar, parity, abort_flag, status, w.wait_ns);
            return __all_sync(0xffffffffu, got);
        };
        const int ew = warp - 2;       // epilogue warp index 0..7
        const int q = warp & 3;        // TMEM lane quarter (fixed by the warp's rank in its warpgroup)
        const int h = ew >> 2;         // column half
        uint32_t* cmw = cms + ew * HALF;   // candidate masks of one tile, [HALF / 32][32 lanes]
        uint32_t* tcmw = tcms + ew * HALF; // column-direction candidate masks
        float* xrow = xch + (size_t)(q * 32 + lane) * kMaxScales * 2;
        uint32_t tcount = 0, npre = 0, nitem = 0;
        bool ok = true;
        for (int idx = it_begin; idx < it_end && ok; ++idx, ++nitem) {
            const Consts<float>* kp; const Bufs<float>* bp; const CUtensorMap* ma; const CUtensorMap* mb;
            long long i0;
            int t0, t1, split, nsplit, nk, nk1;
            item_kb(idx, kp, bp, ma, mb, i0, t0, t1, split, nsplit, nk, nk1);
            const Consts<float>& k = *kp;
            const Bufs<float>& b = *bp;
            const bool pre = nk1 < nk;
            const float T = logf((float)k.n) + 20.0f;
            const long long i = i0 + q * 32 + lane;
            const bool in_range = i < k.n;
            const bool live = in_range && !b.mask[i];
            float nu_i = 0.f, nu1_i = 0.f, nf_i = 0.f, li = -INFINITY;
            if (in_range) {
                nu_i = b.nu[i];
                nf_i = b.nf[i];
                li = b.logw[i];
                if (pre) {   // same summation order as colprep's tc_q1
                    const float* nc = b.nu_chunk + (size_t)i * (k.r_pad / 64);
                    const int c64 = stage_chunks64(k, nk1);
                    for (int c = 0; c < c64; ++c) nu1_i += nc[c];
                }
            }
            const float Fi = sqrtf(nf_i);
            const float rnu_i = sqrt_up(nu_i), rnu1_i = sqrt_up(nu1_i);
            float rowc[N], mx[N], sm[N];
            // the exact self term (u_i - u_i = 0) is the screening reference of every split
            // and of both halves; it is counted once, by the first half of the split whose
            // source range holds i
            const bool self_here = h == 0 && (i / BN) >= t0 && (i / BN) < t1;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                rowc[j] = -0.5f * k.tau[j] * nf_i;
                const bool self = live && li != -INFINITY;
                mx[j] = self ? rowc[j] + li : -INFINITY;
                sm[j] = (self && self_here) ? 1.f : 0.f;
            }
            unsigned long long ncand = 0;
            int exact1 = 0;   // first-pass exact evaluations of this warp in this item
            const uint32_t par = npre & 1u;
            uint32_t* myesc = escm + (ew * 2 + par) * kEscWords;
            if (pre) {
                ++npre;
                for (int wd = lane; wd < kEscWords; wd += 32) myesc[wd] = 0u;
                __syncwarp();
            }
            // one exact score of this lane's row against source src
            // the largest log-weight and source norms over the item's source range (both
            // halves of every tile), for an upper bound of every tile's threshold
            float it_lmax = -INFINITY, it_numax = 0.f, it_numax1 = 0.f;
            {
                const int ca = (int)(((long long)t0 * BN) / 128), cb = (int)(((long long)t1 * BN) / 128);
                for (int c = ca + lane; c < cb; c += 32) {
                    it_lmax = fmaxf(it_lmax, b.tc_tile_lmax[c]);
                    it_numax = fmaxf(it_numax, b.tc_tile_numax[c]);
                    it_numax1 = fmaxf(it_numax1, b.tc_tile_numax1[c]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    it_lmax = fmaxf(it_lmax, __shfl_xor_sync(0xffffffffu, it_lmax, o));
                    it_numax = fmaxf(it_numax, __shfl_xor_sync(0xffffffffu, it_numax, o));
                    it_numax1 = fmaxf(it_numax1, __shfl_xor_sync(0xffffffffu, it_numax1, o));
                }
            }
            const float it_rnumax = sqrt_up(it_numax), it_rnumax1 = sqrt_up(it_numax1);
            float th_hi0 = 0.f, th_hi1 = 0.f;   // the bound over all / first-pass coordinates
            int th_ok = 0;                      // bit fp: th_hi<fp> is current
            // the first test is kept while it settles most chunks of 32 columns (warp-uniform
            // counts): where the screen's margin is thin (low r) it would mostly be work
            // on top of the exact test
            bool use_l0 = true;
            int l0_chunks = 0, l0_pass = 0;
            auto add_score = [&](float s1, float s2, long long src) {
                const float ls = b.mask[src] ? -INFINITY : b.logw[src];
                if (ls == -INFINITY) return;
                th_ok = 0;   // the row maxima may grow
#pragma unroll
                for (int j = 0; j < N; ++j) {
                    const float sc = fmaf(-s1, k.inv2tau[j], s2) + (rowc[j] + ls);
                    if (sc > mx[j]) {
                        sm[j] = (mx[j] == -INFINITY) ? 1.f : sm[j] * expf(mx[j] - sc) + 1.f;
                        mx[j] = sc;
                    } else {
                        sm[j] += expf(sc - mx[j]);
                    }
                }
            };
            // long rows: the warp evaluates the candidates of its 32 rows one at a time,
            // coalesced over the coordinates
            auto eval_warp = [&](uint32_t cm, long long sb) {
                while (true) {
                    const uint32_t who = __ballot_sync(0xffffffffu, cm != 0u);
                    if (who == 0u) break;
                    const int leader = __ffs(who) - 1;
                    const int c = __shfl_sync(0xffffffffu, __ffs(cm) - 1, leader);
                    const long long src = sb + c;
                    const long long tgt = i0 + q * 32 + leader;
                    float s1, s2;
                    pair_sums_warp(k, b, tgt, src, lane, s1, s2);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                    }
                    if (lane == leader) {
                        add_score(s1, s2, src);
                        cm &= cm - 1u;
                        ++ncand;
                    }
                }
            };
            // this warp is done with accumulator acc and q buffer qs
            auto release = [&](int acc, int qs) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&qempty[qs]);
                    // the TMEM loads completed (wait::ld) and are fenced before this signal
                    if (PAIR) mbar_arrive_remote(tpair_lead + (uint32_t)(acc * 8));
                    else mbar_arrive(&tempty[acc]);
                }
            };
            // column direction of a symmetric block: target c (a column) from source i (a
            // row of this item); exact score with the drift at the target, added to the
            // target's accumulator word
            const bool src_live = live && li != -INFINITY;
            auto eval_warp_t = [&](uint32_t cm, long long sb) {
                while (true) {
                    const uint32_t who = __ballot_sync(0xffffffffu, cm != 0u);
                    if (who == 0u) break;
                    const int leader = __ffs(who) - 1;
                    const int c = __shfl_sync(0xffffffffu, __ffs(cm) - 1, leader);
                    const long long tgt = sb + c;
                    const long long src = i0 + q * 32 + leader;
                    float s1, s2;
                    pair_sums_warp(k, b, tgt, src, lane, s1, s2);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                    }
                    if (lane == leader) {
                        const float nft = b.nf[tgt];
#pragma unroll
                        for (int j = 0; j < N; ++j) {
                            const float sc = fmaf(-s1, k.inv2tau[j], s2) + (-0.5f * k.tau[j] * nft + li);
                            lse_atomic_add(&b.tc_xlse[(size_t)tgt * kMaxScales + j], sc, status);
                        }
                        cm &= cm - 1u;
                        ++ncand;
                    }
                }
            };
            const long long a_chunk = i0 / 128;   // the item's target tile as a chunk of 128
            // one tile: mode 0 = single full pass, 1 = first pass, 2 = second pass of a tile
            // this warp marked, 3 = second pass of a tile only other warps marked.  In a
            // symmetric screen this warp's 128-column chunk c is skipped when c < a_chunk
            // (its pairs belong to the block with the roles swapped), screened for this
            // item's rows only when c = a_chunk, and screened in both directions when
            // c > a_chunk.
            auto tile = [&](int t, int mode) -> bool {
                const int acc = (int)(tcount & 1u);
                const uint32_t aph = (tcount >> 1) & 1u;
                const int qs = (int)(tcount % QB);
                const uint32_t qph = (tcount / QB) & 1u;
                ++tcount;
                const long long c0 = (long long)t * BN + h * HALF;   // first source of this warp
                const long long cchunk = c0 / 128;
                const int hm = !k.tc_sym ? 1 : (cchunk < a_chunk ? 0 : (cchunk == a_chunk ? 1 : 2));
                if (mode == 3 || hm == 0) {
                    // unused here, but a q buffer is handed back only once its copy landed (the
                    // producer re-arms its barrier next)
                    if (!wait_warp(&qfull[qs], qph)) return false;
                    if (!wait_warp(&tfull[acc], aph)) return false;
                    tc_fence_after();
                    release(acc, qs);
                    return true;
                }
                const bool first_pass = (mode == 1);
                const float nu_s = first_pass ? nu1_i : nu_i;
                // this warp's columns of the staged q values and the tile's chunk maxima
                // (producer, per tile, q buffer qs)
                const float* qw = qbuf + qs * BN + h * HALF;
                const float* qtw = qtbuf + qs * BN + h * HALF;   // q_c - (rho_c^2 + err_c)
                const float* ci = qinfo + qs * 16;
                if (!wait_warp(&qfull[qs], qph)) return false;
                const float rnu_s = first_pass ? rnu1_i : rnu_i;
                // the tile's threshold, from its chunk maxima
                auto tile_theta = [&]() -> float {
                    float lmax = ci[0];
                    float numax = first_pass ? ci[2] : ci[1];
                    float rnumax = first_pass ? ci[6] : ci[5];
                    if (BN == 256) {
                        lmax = fmaxf(lmax, ci[8]);
                        numax = fmaxf(numax, first_pass ? ci[10] : ci[9]);
                        rnumax = fmaxf(rnumax, first_pass ? ci[14] : ci[13]);
                    }
                    return screen_theta<N>(k, live, nu_s, rnu_s, Fi, mx, lmax, numax, rnumax, T);
                };
                const float nu_src = (hm == 2 && src_live) ? nu_s : INFINITY;
                // one test per lane and 32 columns covers both directions: a pair can be a
                // candidate only if q_s - 2 G <= max(theta_i, Rmax - nu_i), Rmax the largest
                // column bound of this warp's chunk
                const float rmax_c = ci[(BN == 256 ? h : 0) * 8 + (first_pass ? 4 : 3)];
                if (!wait_warp(&tfull[acc], aph)) return false;
                tc_fence_after();
                const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + h * HALF);
                if (k.r <= 64) {
                    // short rows (one pass, no symmetric blocks): every lane evaluates its own
                    // row's candidates chunk by chunk, tightening the screen as the running
                    // maxima grow
                    const float* ut = b.u + (size_t)i * k.r_pad;
                    float theta = tile_theta();
                    for (int ch = 0; ch < HALF / 32; ++ch) {
                        uint32_t v[32];
                        __syncwarp();
                        tmem_ld32(tbase + (uint32_t)(ch * 32), v);
                        tmem_ld_wait();
                        uint32_t cm = 0;
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const float dd = fmaf(k.tc_g2, __uint_as_float(v[c]), qw[ch * 32 + c]);
                            cm |= (dd <= theta ? 1u : 0u) << c;
                        }
                        const long long sb = c0 + ch * 32;
                        if (i >= sb && i < sb + 32) cm &= ~(1u << (int)(i - sb));   // self term already counted
                        while (cm) {
                            const int c = __ffs(cm) - 1;
                            cm &= cm - 1u;
                            const long long src = sb + c;
                            const float* us = b.u + (size_t)src * k.r_pad;
                            float s1 = 0.f, s2 = 0.f;
                            for (int d = 0; d < k.r; ++d) {
                                const float dl = ut[d] - us[d];
                                s1 = fmaf(dl, dl, s1);
                                s2 = fmaf(dl, drift_at(k, b, i, ut[d], d), s2);
                            }
                            add_score(s1, s2, src);
                            ++ncand;
                        }
                        theta = tile_theta();
                    }
                    release(acc, qs);
                    return true;
                }
                // long rows: 32 columns per TMEM load.  First test: with q_min the smallest
                // q_s of the 32 columns and a_max the largest accumulator, q_min + g2 a_max
                // (g2 < 0) is below every column's q_s - 2 G up to rounding, which the margin
                // covers; only a lane that passes it (some lane of the warp) computes the
                // smallest q_s - 2 G, and only when that passes theta_any the candidate masks
                int cnt = 0;
                const float* qmw = qmbuf + qs * (BN / 32) + h * (HALF / 32);
                // the threshold from the item's maxima bounds every tile's from above
                // (screen_theta grows with lmax, numax and rnumax; the margin covers
                // rounding); the tile's own is computed only for a lane that passes with it
                const int fp = first_pass ? 1 : 0;
                if (use_l0 && !(th_ok & (1 << fp))) {
                    const float th = screen_theta<N>(k, live, nu_s, rnu_s, Fi, mx, it_lmax, fp ? it_numax1 : it_numax,
                                                     fp ? it_rnumax1 : it_rnumax, T);
                    const float thm = (th == -INFINITY) ? th : th + 1e-6f * (fabsf(th) + nu_s + 1.f);
                    if (fp) th_hi1 = thm; else th_hi0 = thm;
                    th_ok |= 1 << fp;
                }
                const float th_hi = fp ? th_hi1 : th_hi0;
                const float tany_hi = (hm == 2 && src_live) ? fmaxf(th_hi, rmax_c - nu_src) : th_hi;
                float theta = 0.f, theta_any = 0.f;
                bool have_theta = false;
                if (!use_l0) {
                    theta = tile_theta();
                    theta_any = (hm == 2 && src_live) ? fmaxf(theta, rmax_c - nu_src) : theta;
                    have_theta = true;
                }
                uint32_t nzm = 0;
                for (int ch = 0; ch < HALF / 32; ++ch) {
                    uint32_t v[32];
                    __syncwarp();
                    tmem_ld32(tbase + (uint32_t)(ch * 32), v);
                    tmem_ld_wait();
                    if (use_l0) {
                        float am0 = __uint_as_float(v[0]), am1 = __uint_as_float(v[1]);
#pragma unroll
                        for (int c = 2; c < 32; c += 4) {
                            am0 = fmax3(am0, __uint_as_float(v[c]), __uint_as_float(v[c + 1]));
                            if (c + 3 < 32) am1 = fmax3(am1, __uint_as_float(v[c + 2]), __uint_as_float(v[c + 3]));
                        }
                        const float qm = qmw[ch];
                        const float g2a = k.tc_g2 * fmaxf(am0, am1);
                        const float l0 = qm + g2a;
                        const float l0m = 1e-6f * (fabsf(qm) + fabsf(g2a));
                        bool pass = l0 <= tany_hi + (l0m + 1e-6f * fabsf(tany_hi));
                        ++l0_chunks;
                        l0_pass += __any_sync(0xffffffffu, pass) ? 1 : 0;
                        if (pass) {
                            if (!have_theta) {
                                theta = tile_theta();
                                theta_any = (hm == 2 && src_live) ? fmaxf(theta, rmax_c - nu_src) : theta;
                                have_theta = true;
                            }
                            pass = l0 <= theta_any + (l0m + 1e-6f * fabsf(theta_any));
                        }
                        if (!pass) continue;
                    }
                    const float4* q4 = reinterpret_cast<const float4*>(qw + ch * 32);
                    // q_s - 2 G two columns per packed FMA, folded into two independent
                    // minimum chains by three-input minima
                    const float2 g2v = make_float2(k.tc_g2, k.tc_g2);
                    float m0c = INFINITY, m1c = INFINITY;
#pragma unroll
                    for (int c4 = 0; c4 < 8; ++c4) {
                        const float4 qq = q4[c4];
                        const float2 d01 = ffma2(g2v, make_float2(__uint_as_float(v[4 * c4 + 0]), __uint_as_float(v[4 * c4 + 1])),
                                                 make_float2(qq.x, qq.y));
                        const float2 d23 = ffma2(g2v, make_float2(__uint_as_float(v[4 * c4 + 2]), __uint_as_float(v[4 * c4 + 3])),
                                                 make_float2(qq.z, qq.w));
                        m0c = fmin3(m0c, d01.x, d01.y);
                        m1c = fmin3(m1c, d23.x, d23.y);
                    }
                    const float mn = fminf(m0c, m1c);
                    uint32_t m0 = 0, t0m = 0;
                    if (mn <= theta_any) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const float g2 = k.tc_g2 * __uint_as_float(v[c]);
                            m0 |= (g2 + qw[ch * 32 + c] <= theta ? 1u : 0u) << c;
                            if (hm == 2) t0m |= ((g2 + qtw[ch * 32 + c]) + nu_src <= 0.f ? 1u : 0u) << c;
                        }
                        const long long sb = c0 + ch * 32;   // self term already counted
                        if (i >= sb && i < sb + 32) m0 &= ~(1u << (int)(i - sb));
                        cnt += __popc(m0) + __popc(t0m);
                    }
                    if (m0 | t0m) {   // masks are stored only where nonzero (bit ch of nzm)
                        cmw[ch * 32 + lane] = m0;
                        tcmw[ch * 32 + lane] = t0m;
                        nzm |= 1u << ch;
                    }
                }
                release(acc, qs);
                if (use_l0 && l0_chunks >= 16 && 2 * l0_pass > l0_chunks) use_l0 = false;
                const int tot = (int)__reduce_add_sync(0xffffffffu, (unsigned)cnt);
                if (tot == 0) return true;
                if (first_pass && (tot > kEscThresh || exact1 + tot > kExactBudget)) {
                    if (lane == 0) myesc[(t - t0) >> 5] |= 1u << ((t - t0) & 31);
                    return true;
                }
                if (first_pass) exact1 += tot;
                for (int ch = 0; ch < HALF / 32; ++ch)
                    eval_warp(((nzm >> ch) & 1u) ? cmw[ch * 32 + lane] : 0u, c0 + ch * 32);
                if (hm == 2)
                    for (int ch = 0; ch < HALF / 32; ++ch)
                        eval_warp_t(((nzm >> ch) & 1u) ? tcmw[ch * 32 + lane] : 0u, c0 + ch * 32);
                return true;
            };
            for (int t = t0; t < t1 && ok; ++t) ok = tile(t, pre ? 1 : 0);
            if (ok && pre) {
                __syncwarp();
                if (lane == 0) {
                    if (PAIR) {   // this warp's marks are read by both CTAs
                        mbar_arrive_cluster(mapa_shared(escb, rank));
                        mbar_arrive_cluster(escb_peer);
                    } else {
                        mbar_arrive(escb);
                    }
                }
                if (!wait_warp(escb, par, CL)) ok = false;
                for (int t = t0; t < t1 && ok; ++t)
                    if (esc_any(par, t - t0)) ok = tile(t, esc_bit(ew, par, t - t0) ? 2 : 3);
            }
            // merge the pair's row states: the second half hands its (max, sum) over through
            // shared memory (bounded hand-shakes, so an aborted partner cannot block)
            const uint32_t xph = nitem & 1u;
            if (ok && h == 1) {
                if (nitem > 0 && !wait_warp(&xfree[q], xph ^ 1u)) ok = false;
                if (ok) {
#pragma unroll
                    for (int j = 0; j < N; ++j) { xrow[2 * j] = mx[j]; xrow[2 * j + 1] = sm[j]; }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&xfull[q]);
                }
            }
            if (ok && h == 0) {
                if (!wait_warp(&xfull[q], xph)) ok = false;
                if (ok) {
#pragma unroll
                    for (int j = 0; j < N; ++j) {
                        const float m2 = xrow[2 * j], s2 = xrow[2 * j + 1];
                        if (s2 > 0.f) {
                            if (sm[j] == 0.f) { mx[j] = m2; sm[j] = s2; }
                            else if (m2 > mx[j]) { sm[j] = sm[j] * expf(mx[j] - m2) + s2; mx[j] = m2; }
                            else sm[j] += s2 * expf(m2 - mx[j]);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&xfree[q]);
                    if (in_range) {
                        if (nsplit == 1 && !k.tc_sym) {
                            b.logw_pred[i] = live ? combine_scales<float, N>(k, mx, sm, b.divf[i], li,
                                                                             b.stats->c_ref, &b.stats->clamps)
                                                  : -INFINITY;
                        } else {
#pragma unroll
                            for (int j = 0; j < N; ++j) {
                                float* ps = part_slot(b, i, split, j);
                                ps[0] = (sm[j] > 0.f) ? mx[j] : -INFINITY;
                                ps[1] = sm[j];
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ncand += __shfl_xor_sync(0xffffffffu, ncand, o);
            if (lane == 0 && ncand) atomicAdd(&b.stats->candidates, ncand);
        }
    }
    tc_fence_before();
    __syncthreads();
    // a pair leaves together: no remote arrive, mark read or MMA into this CTA's TMEM is
    // outstanding once both CTAs are here
    if (PAIR) cluster_sync();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        if (PAIR) tmem_dealloc_pair(tmem, C::TMEM_COLS);
        else tmem_dealloc(tmem, C::TMEM_COLS);
    }
    // the last CTA to finish runs the first-pass controller of every filter of the launch
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int prev = atomicAdd(&ctr->tc_done, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            if (!batched) {
                tc_adapt(k0, b0.stats);
            } else {
                for (int f = 0; f < w.nb; ++f)
                    if (w.tr[f].path == 0) tc_adapt(w.tr[f].k, w.tr[f].b.stats);
            }
            atomicExch(&ctr->tc_done, 0u);
        }
    }
}

// Combines the split states of every row (and, for the symmetric screen, the terms the row
// received as a column) and applies the multi-scale combination.
template <int N>
__device__ __forceinline__ void tc_merge_body(const Consts<float>& k, const Bufs<float>& b, int nsplit, int bid, int nblk) {
    if (nsplit <= 1 && !k.tc_sym) return;
    const int nst = (int)(k.n_pad / 256);
    for (long long i = k.row0 + bid * (long long)blockDim.x + threadIdx.x; i < k.row1; i += (long long)nblk * blockDim.x) {
        if (b.mask[i]) { b.logw_pred[i] = -INFINITY; continue; }
        const int ns = k.tc_sym ? tc_sym_splits(nst - (int)(i / 256), k.tc_split_len) : nsplit;
        float mx[N], sm[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
            float m = -INFINITY, s = 0.f;
            auto add = [&](float m2, float s2) {
                if (m2 == -INFINITY || !(s2 > 0.f)) return;
                if (m == -INFINITY) { m = m2; s = s2; }
                else if (m2 > m) { s = s * expf(m - m2) + s2; m = m2; }
                else s += s2 * expf(m2 - m);
            };
            for (int q = 0; q < ns; ++q) {
                const float* ps = part_slot(b, i, q, j);
                add(ps[0], ps[1]);
            }
            if (k.tc_sym) {
                const unsigned long long w = b.tc_xlse[(size_t)i * kMaxScales + j];
                add(__uint_as_float((uint32_t)w), __uint_as_float((uint32_t)(w >> 32)));
            }
            mx[j] = m;
            sm[j] = s;
        }
        b.logw_pred[i] = combine_scales<float, N>(k, mx, sm, b.divf[i], b.logw[i], b.stats->c_ref, &b.stats->clamps);
    }
}

template <int N>
__global__ void k_tc_merge(Consts<float> k, Bufs<float> b, int nsplit) { tc_merge_body<N>(k, b, nsplit, blockIdx.x, gridDim.x); }

template <int N>
__global__ void kb_tc_merge(const Traj<float>* __restrict__ tr) {
    const Traj<float>& t = tr[blockIdx.y];
    if (t.path != 0) return;
    tc_merge_body<N>(t.k, t.b, t.b.tc_splits, blockIdx.x, gridDim.x);
}

size_t tc_scratch_bytes(long long n_pad) {
    return (size_t)n_pad * sizeof(float) + 2 * (size_t)(n_pad / 128) * sizeof(float) +
           (size_t)n_pad * kMaxSplit * kMaxScales * 2 * sizeof(float) + 2048;
}

// Split count of a single filter's prediction: minimises the makespan
// ceil(tiles * S / grid) * (source tiles / S + overhead) over S = 1..8.
int tc_choose_splits(long long tiles, int nst, int grid) {
    int best = 1;
    double best_t = INFINITY;
    for (int S = 1; S <= kMaxSplit && S <= nst; ++S) {
        const double waves = (double)((tiles * S + grid - 1) / grid);
        const double t = waves * ((double)nst / S + 2.0);
        if (t < best_t - 1e-9) { best_t = t; best = S; }
    }
    return best;
}

int tc_max_split() { return kMaxSplit; }

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

template <int BN, bool PAIR>
cudaError_t set_attr_all() {
    cudaError_t e = cudaSuccess;
    const int sm = tc::Cfg<BN, PAIR>::SMEM_BYTES;
    // the block must be launchable at its size (registers per thread x threads)
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, k_ksum_tc<3, BN, PAIR>)) != cudaSuccess) return e;
    if (fa.maxThreadsPerBlock < tc::NUM_THREADS) return cudaErrorLaunchOutOfResources;
    const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ksum_tc<1, BN, PAIR>, a, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ksum_tc<2, BN, PAIR>, a, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ksum_tc<3, BN, PAIR>, a, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ksum_tc<4, BN, PAIR>, a, sm);
    return e;
}

template <int BN>
cudaError_t launch_bn(int N, unsigned grid, const CUtensorMap& a, const CUtensorMap& bm, const Consts<float>& k,
                      const Bufs<float>& b, const TcWork& w, cudaStream_t s) {
    if (grid == 0) return cudaSuccess;
    const int sm = tc::Cfg<BN>::SMEM_BYTES;
    switch (N) {
        case 1: k_ksum_tc<1, BN, false><<<grid, tc::NUM_THREADS, sm, s>>>(a, bm, k, b, w); break;
        case 2: k_ksum_tc<2, BN, false><<<grid, tc::NUM_THREADS, sm, s>>>(a, bm, k, b, w); break;
        case 3: k_ksum_tc<3, BN, false><<<grid, tc::NUM_THREADS, sm, s>>>(a, bm, k, b, w); break;
        case 4: k_ksum_tc<4, BN, false><<<grid, tc::NUM_THREADS, sm, s>>>(a, bm, k, b, w); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Launch configuration of the pair kernel: `clusters` 2-CTA clusters, one CTA per SM.
cudaLaunchConfig_t pair_config(unsigned clusters, cudaStream_t s, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters);
    cfg.blockDim = dim3(tc::NUM_THREADS);
    cfg.dynamicSmemBytes = tc::Cfg<256, true>::SMEM_BYTES;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}
template <int N>
cudaError_t launch_pair_n(unsigned clusters, const CUtensorMap& a, const Consts<float>& k, const Bufs<float>& b,
                          const TcWork& w, cudaStream_t s) {
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = pair_config(clusters, s, at);
    return cudaLaunchKernelEx(&cfg, k_ksum_tc<N, 256, true>, a, a, k, b, w);
}
cudaError_t launch_pair(int N, unsigned clusters, const CUtensorMap& a, const Consts<float>& k, const Bufs<float>& b,
                        const TcWork& w, cudaStream_t s) {
    if (clusters == 0) return cudaSuccess;
    switch (N) {
        case 1: return launch_pair_n<1>(clusters, a, k, b, w, s);
        case 2: return launch_pair_n<2>(clusters, a, k, b, w, s);
        case 3: return launch_pair_n<3>(clusters, a, k, b, w, s);
        case 4: return launch_pair_n<4>(clusters, a, k, b, w, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// TMA map of the screen's operand copy: rows x cols elements, bf16 (box 64 x box_rows) or
// e4m3 bytes (box 128 x box_rows), 128-byte swizzle either way.
bool make_tc_map(void* map_out, const void* base, long long rows, int cols, int box_rows, bool fp8) {
    CUtensorMap* map = static_cast<CUtensorMap*>(map_out);
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * (fp8 ? 1 : 2)};
    const cuuint32_t box[2] = {(cuuint32_t)(fp8 ? 128 : tc::BK), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
              dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Opts the prediction kernels into their shared-memory size on the current device (called
// when a BF16 handle or batch is created, so that no attribute call happens during
// stream capture).
cudaError_t prepare_ksum_tc() {
    cudaError_t e = set_attr_all<256, false>();
    if (e == cudaSuccess) e = set_attr_all<128, false>();
    if (e == cudaSuccess) e = set_attr_all<256, true>();
    return e;
}

// How many 2-CTA clusters of the pair kernel can be resident at once on the current
// device (0 when clusters of its size cannot be placed).  Host-side set-up only.
int tc_pair_max_clusters() {
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = pair_config(1, nullptr, at);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_ksum_tc<3, 256, true>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

// Single filter: the work list (items, cta_start) was built by the handle
// (yy_api.cu::build_tc_schedule) in the filter's workspace; nsplit source splits.
cudaError_t launch_ksum_tc(const Consts<float>& k, const Bufs<float>& b, cudaStream_t s, int* launches) {
    if (!b.ubf || !b.tc_items || k.n_pad % 256 != 0 || k.r_pad % tc::BK != 0) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    const int cols = k.tc_fp8 ? k.tc_r8 : k.r_pad;
    if (!make_tc_map(&ma, b.ubf, k.n_pad, cols, tc::BM, k.tc_fp8) || !make_tc_map(&mb, b.ubf, k.n_pad, cols, 256, k.tc_fp8))
        return cudaErrorNotSupported;
    cudaError_t e = cudaMemsetAsync(&b.stats->candidates, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_tc_colprep<<<(unsigned)(k.n_pad / 128), 128, 0, s>>>(k, b);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (k.tc_sym) {
        k_tc_colprep2<<<(unsigned)(k.n_pad / 128), 128, 0, s>>>(k, b);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const TcWork w{nullptr, nullptr, b.tc_items, b.tc_cta_start, 1, k.wait_ns};
    // tc_grid counts CTAs; a paired schedule has tc_grid / 2 work lists, one per cluster
    e = b.tc_pair ? launch_pair(k.N, (unsigned)(b.tc_grid / 2), ma, k, b, w, s)
                  : launch_bn<256>(k.N, (unsigned)b.tc_grid, ma, mb, k, b, w, s);
    if (e != cudaSuccess) return e;
    int l = k.tc_sym ? 3 : 2;
    if (b.tc_splits > 1 || k.tc_sym) {
        const unsigned g = (unsigned)std::min<long long>((k.n + 255) / 256, 1024);
        switch (k.N) {
            case 1: k_tc_merge<1><<<g, 256, 0, s>>>(k, b, b.tc_splits); break;
            case 2: k_tc_merge<2><<<g, 256, 0, s>>>(k, b, b.tc_splits); break;
            case 3: k_tc_merge<3><<<g, 256, 0, s>>>(k, b, b.tc_splits); break;
            case 4: k_tc_merge<4><<<g, 256, 0, s>>>(k, b, b.tc_splits); break;
        }
        l += 1;
    }
    if (launches) *launches += l;
    return cudaGetLastError();
}

// Batched prediction: column preparation for every filter, then one persistent launch
// over the precomputed item lists.  bn selects the source-tile width (256 or 128).
cudaError_t launch_ksum_tc_batch(const Traj<float>* d_traj, int B, int N, long long n_pad_max,
                                 const void* d_maps, const int4* d_items, const int* d_cta_start,
                                 int grid, int bn, const Consts<float>& k_any, const Bufs<float>& b_any,
                                 const void* map_any_v, cudaStream_t s, int* launches) {
    kb_tc_colprep<<<dim3((unsigned)(n_pad_max / 128), B), 128, 0, s>>>(d_traj);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const CUtensorMap& map_any = *static_cast<const CUtensorMap*>(map_any_v);
    const TcWork w{d_traj, static_cast<const CUtensorMap*>(d_maps), d_items, d_cta_start, B, k_any.wait_ns};
    e = (bn == 128) ? launch_bn<128>(N, (unsigned)grid, map_any, map_any, k_any, b_any, w, s)
                    : launch_bn<256>(N, (unsigned)grid, map_any, map_any, k_any, b_any, w, s);
    if (e != cudaSuccess) return e;
    const dim3 mg((unsigned)std::min<long long>((n_pad_max + 255) / 256, 256), B);
    switch (N) {
        case 1: kb_tc_merge<1><<<mg, 256, 0, s>>>(d_traj); break;
        case 2: kb_tc_merge<2><<<mg, 256, 0, s>>>(d_traj); break;
        case 3: kb_tc_merge<3><<<mg, 256, 0, s>>>(d_traj); break;
        case 4: kb_tc_merge<4><<<mg, 256, 0, s>>>(d_traj); break;
    }
    if (launches) *launches += 3;
    return cudaGetLastError();
}

}  // namespace yy
