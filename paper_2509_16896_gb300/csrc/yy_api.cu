// C ABI of libyy (declared in include/yy.h): argument checks, workspace carving, host
// constants (multi-scale coefficients, offsets) and the launch sequences.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "yy_handle.cuh"

using namespace yy;

namespace {

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

constexpr int kMaxTcGrid = 1024;
constexpr unsigned long long kDefaultWaitNs = 4000000000ull;   // 4 s

// Work list of the single-filter BF16 prediction: one persistent CTA per SM.  Symmetric
// screen (the usual case): target tile a (128 rows) covers the source tiles from the one
// holding row 128 a on (L_a = nst - a / 2 tiles of 256), split into tc_sym_splits(L_a)
// ranges; items are assigned longest first to the least loaded CTA.  Otherwise every
// target tile is split into S ranges (S minimising the makespan) dealt round-robin.
// CTA pairs (when allowed, the handle's first row starts a 256-row super-tile -- always:
// shard chunks are whole super-tiles -- and the device can place 2-CTA clusters): the same
// construction over super-tiles p (target tiles 2p and 2p + 1, both with L = nst - p), one
// work list per cluster.  A last tile of odd index gets its pair partner from the padding
// rows (n_pad is a multiple of 256), which the kernel treats as out of range.
// Copied into the workspace; synchronous (set-up only).
yy_status build_tc_schedule(yy_filter* f) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the handle's target tiles (all of them, or its shard's chunk)
    long long t_lo = f->row0 / 128, t_hi = (f->row1 + 127) / 128;
    const int max_cl = f->pair_ok ? tc_pair_max_clusters() : 0;
    const bool pair = max_cl > 0 && t_lo % 2 == 0 && (t_hi + 1) / 2 * 256 <= f->n_pad;
    const int span = pair ? 2 : 1;   // target tiles per item
    const int units = pair ? std::min(max_cl, sms / 2) : std::min(sms, kMaxTcGrid);
    if (pair) { t_lo /= 2; t_hi = (t_hi + 1) / 2; }   // super-tiles
    const long long tiles = t_hi - t_lo;
    const int nst = (int)(f->n_pad / 256);
    const int grid = (int)std::min<long long>(units, tiles * 8);
    std::vector<std::vector<int4>> per(grid);
    int S = 1;
    if (f->kf.tc_sym) {
        // range length: 64 source tiles, or shorter (down to 8) where a CTA's share of the
        // blocks is small, so that every CTA gets about four items to balance with; taken
        // per CTA (a cluster holds two), so that both forms split alike and take the same
        // screening decisions
        double work = 0.0;
        for (long long t = t_lo; t < t_hi; ++t) work += span * (double)(nst - (int)(span == 2 ? t : t / 2));
        const int ctas = span * grid;
        const int len = (int)std::max(8.0, std::min(64.0, work / ctas / 4.0));
        f->kf.tc_split_len = len;
        struct It { double cost; int t, q, S; };
        std::vector<It> all;
        for (long long t = t_lo; t < t_hi; ++t) {
            const int L = nst - (int)(span == 2 ? t : t / 2);
            const int St = tc_sym_splits(L, len);
            for (int q = 0; q < St; ++q)
                all.push_back({(double)((L * (q + 1)) / St - (L * q) / St) + 1.0, (int)t, q, St});
            S = std::max(S, St);
        }
        std::stable_sort(all.begin(), all.end(), [](const It& x, const It& y) { return x.cost > y.cost; });
        std::vector<double> load(grid, 0.0);
        for (const It& it : all) {
            const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            per[c].push_back(make_int4(0, it.t, it.q, it.S));
            load[c] += it.cost;
        }
    } else {
        S = tc_choose_splits(tiles, nst, std::max(grid, 1));
        long long j = 0;
        for (long long t = t_lo; t < t_hi; ++t)
            for (int q = 0; q < S; ++q, ++j) per[j % grid].push_back(make_int4(0, (int)t, q, S));
    }
    std::vector<int4> items;
    std::vector<int> start(grid + 1);
    for (int c = 0; c < grid; ++c) {
        start[c] = (int)items.size();
        items.insert(items.end(), per[c].begin(), per[c].end());
    }
    start[grid] = (int)items.size();
    cudaError_t e = cudaMemcpyAsync(f->bf.tc_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                                    f->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f->bf.tc_cta_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice,
                            f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    f->bf.tc_grid = pair ? 2 * grid : grid;   // CTAs
    f->bf.tc_splits = S;
    f->bf.tc_pair = pair ? 1 : 0;
    return YY_OK;
}

}  // namespace

namespace yy {
yy_status rebuild_tc_schedule(yy_filter* f) { return build_tc_schedule(f); }
}  // namespace yy

namespace {

bool cfg_valid(const yy_config* c) {
    if (!c) return false;
    if (c->r < 1 || c->r > YY_MAX_DIM || c->m != c->r) return false;
    if (c->n < 2 || c->n > (1LL << 31)) return false;
    if (!(c->dt > 0.0) || !(c->R > 0.0) || !(c->prior_var > 0.0)) return false;
    if (c->n_scales < 1 || c->n_scales > YY_MAX_SCALES) return false;
    if (c->model != YY_MODEL_CUBIC && c->model != YY_MODEL_LINEAR && c->model != YY_MODEL_PAPER_E1) return false;
    if (c->precision < YY_PREC_FP64 || c->precision > YY_PREC_FP32_SCREEN) return false;
    if (c->restart_init != YY_RESTART_INIT_GAUSS && c->restart_init != YY_RESTART_INIT_UNIFORM) return false;
    if (!(c->ess_frac >= 0.0) || c->ess_frac > 1.0) return false;
    if (c->restart_rule != YY_RESTART_PLAIN && c->restart_rule != YY_RESTART_LEARNED) return false;
    if (c->screen_prefix < 0) return false;
    if (c->screen_type != YY_SCREEN_BF16 && c->screen_type != YY_SCREEN_FP8) return false;
    if (c->noise != YY_NOISE_UNIT && c->noise != YY_NOISE_DIAG) return false;
    if (c->noise == YY_NOISE_DIAG) {
        if (!(c->noise_u > 0.0) || !(c->noise_v > 0.0) || !(c->noise_u_kappa >= 0.0) || !(c->noise_v_kappa >= 0.0))
            return false;
        if (c->noise_u_zero < 0 || c->noise_u_zero > c->r) return false;
    }
    if (c->materialise < 0 || c->materialise > 2) return false;
    return true;
}

// Configurations the library does not run: noise coefficients outside the plain FP32 / FP64
// forms (the screens bound Euclidean distances) or with the large-scale model (its centred
// update does not separate from state-dependent b(x)).
bool cfg_supported(const yy_config* c) {
    if (c->noise == YY_NOISE_DIAG)
        return (c->precision == YY_PREC_FP32 || c->precision == YY_PREC_FP64) && c->model != YY_MODEL_PAPER_E1 &&
               c->materialise == 0;
    if (c->materialise != 0) return c->precision != YY_PREC_FP64;   // the operator is float32
    return true;
}

// Sequential carve of the workspace with 256-byte alignment.
struct Carver {
    char* base;
    size_t off = 0;
    template <typename P>
    P* take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        P* p = base ? reinterpret_cast<P*>(base + off) : nullptr;
        off += bytes;
        return p;
    }
};

template <typename T>
size_t carve(const yy_config* c, char* base, Bufs<T>* out) {
    const long long n_pad = round_up(c->n, kRowAlign);
    const int r_pad = (int)round_up(c->r, kColAlign);
    Carver cv{base};
    Bufs<T> b{};
    const size_t nr = (size_t)n_pad * r_pad;
    b.u = cv.take<float>(nr * sizeof(float));
    b.f = cv.take<T>(nr * sizeof(T));
    // the screen's exact pairs recompute the drift from one coordinate unless f is stored; the
    // large-scale model's drift couples neighbouring coordinates, so it is always stored
    b.store_f = (c->precision == YY_PREC_BF16 && c->model != YY_MODEL_PAPER_E1) ? 0 : 1;
    b.ubf = (c->precision == YY_PREC_BF16) ? cv.take<__nv_bfloat16>(nr * sizeof(__nv_bfloat16)) : nullptr;
    b.divf = cv.take<T>(n_pad * sizeof(T));
    b.nu = cv.take<T>(n_pad * sizeof(T));
    b.nf = cv.take<T>(n_pad * sizeof(T));
    b.mask = cv.take<uint8_t>(n_pad);
    b.logw = cv.take<T>(n_pad * sizeof(T));
    b.logw_pred = cv.take<T>(n_pad * sizeof(T));
    b.centre = cv.take<double>(r_pad * sizeof(double));
    b.halfwidth = cv.take<double>(r_pad * sizeof(double));
    b.mean = cv.take<double>(r_pad * sizeof(double));
    b.var = cv.take<double>(r_pad * sizeof(double));
    b.dirs = cv.take<uint32_t>((size_t)c->r * 33 * sizeof(uint32_t));
    b.params = cv.take<uint32_t>((size_t)c->r * (YY_SOBOL_POLY_WORDS + YY_SOBOL_SCRAMBLE_WORDS) * sizeof(uint32_t));
    b.obs_g = cv.take<T>(r_pad * sizeof(T));
    b.obs_c = cv.take<T>(r_pad * sizeof(T));
    b.obs_l = cv.take<T>(r_pad * sizeof(T));
    b.obs_ibc = cv.take<T>(r_pad * sizeof(T));
    if (c->noise == YY_NOISE_DIAG) {
        b.minv = cv.take<T>(nr * sizeof(T));
        b.hld = cv.take<T>(n_pad * sizeof(T));
    }
    if (c->materialise != 0 && c->precision != YY_PREC_FP64)
    {
        b.op = cv.take<float>((size_t)c->n_scales * (size_t)n_pad * (size_t)n_pad * sizeof(float));
        b.op_lsrc = cv.take<float>((size_t)n_pad * sizeof(float));
    }
    b.dimc = cv.take<T>(5 * (size_t)r_pad * sizeof(T));
    b.next_centre = cv.take<double>(r_pad * sizeof(double));
    b.next_half = cv.take<double>(r_pad * sizeof(double));
    b.dy_last = cv.take<double>(r_pad * sizeof(double));
    b.part = cv.take<double>(part_bytes(r_pad));
    b.part_list = cv.take<int>((size_t)kNumPartBlocks * sizeof(int));
    b.stats = cv.take<DevStats>(sizeof(DevStats));
    if (c->precision == YY_PREC_BF16 || c->precision == YY_PREC_FP32_SCREEN)
        b.nu_chunk = cv.take<float>((size_t)n_pad * (r_pad / kColAlign) * sizeof(float));
    // plain form of a filter with fewer than two target blocks of 64 per SM: its source
    // ranges' partial states
    if ((c->precision == YY_PREC_FP32 || c->precision == YY_PREC_FP64) && n_pad < 2 * 152 * 64)
        b.simt_part = cv.take<T>((size_t)n_pad * kSimtMaxSplit * kMaxScales * 2 * sizeof(T));
    if (c->precision == YY_PREC_BF16) {
        b.tc_q = cv.take<float>((size_t)n_pad * sizeof(float));
        b.tc_q1 = cv.take<float>((size_t)n_pad * sizeof(float));
        b.tc_q1t = cv.take<float>((size_t)n_pad * sizeof(float));
        b.tc_qmin = cv.take<float>((size_t)(n_pad / 32) * sizeof(float));
        b.tc_qmin1 = cv.take<float>((size_t)(n_pad / 32) * sizeof(float));
        b.tc_qt = cv.take<float>((size_t)n_pad * sizeof(float));
        b.tc_qt1 = cv.take<float>((size_t)n_pad * sizeof(float));
        b.tc_tile_rmax = cv.take<float>((size_t)(n_pad / 128) * sizeof(float));
        b.tc_tile_rmax1 = cv.take<float>((size_t)(n_pad / 128) * sizeof(float));
        b.tc_cinfo = cv.take<float>((size_t)(n_pad / 128) * 8 * sizeof(float));
        b.tc_xlse = cv.take<unsigned long long>((size_t)n_pad * kMaxScales * sizeof(unsigned long long));
        b.tc_tile_lmax = cv.take<float>((size_t)(n_pad / 128) * sizeof(float));
        b.tc_tile_numax = cv.take<float>((size_t)(n_pad / 128) * sizeof(float));
        b.tc_tile_numax1 = cv.take<float>((size_t)(n_pad / 128) * sizeof(float));
        b.tc_part = cv.take<float>((size_t)n_pad * 8 * kMaxScales * 2 * sizeof(float));
        b.tc_items = cv.take<int4>((size_t)(n_pad / 128) * 8 * sizeof(int4));
        b.tc_cta_start = cv.take<int>((size_t)(kMaxTcGrid + 1) * sizeof(int));
    }
    if (out) *out = b;
    return cv.off + 256;
}

// Coefficients of eq. general_kernel: V c = d with rows (1..1 | 1), (s_j^-1 | 0),
// (s_j^-mu_k | 0), mu_k = 3/2, 2, ..., solved by Gaussian elimination with partial pivoting.
void multiscale_coefficients(int N, double* c) {
    const int M = N + 1;
    double A[kMaxScales + 1][kMaxScales + 2];
    for (int row = 0; row < M; ++row)
        for (int col = 0; col <= M; ++col) A[row][col] = 0.0;
    for (int j = 0; j < M; ++j) A[0][j] = 1.0;
    A[0][M] = 1.0;
    for (int j = 0; j < N; ++j) A[1][j] = 1.0 / ldexp(1.0, j);
    A[1][M] = 1.0;
    for (int k = 0; k + 2 < M; ++k) {
        const double mu = 1.5 + 0.5 * k;
        for (int j = 0; j < N; ++j) A[2 + k][j] = pow(ldexp(1.0, j), -mu);
    }
    for (int col = 0; col < M; ++col) {
        int piv = col;
        for (int row = col + 1; row < M; ++row)
            if (fabs(A[row][col]) > fabs(A[piv][col])) piv = row;
        if (piv != col)
            for (int q = 0; q <= M; ++q) { double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
        for (int row = col + 1; row < M; ++row) {
            const double f = A[row][col] / A[col][col];
            for (int q = col; q <= M; ++q) A[row][q] -= f * A[col][q];
        }
    }
    for (int row = M - 1; row >= 0; --row) {
        double s = A[row][M];
        for (int q = row + 1; q < M; ++q) s -= A[row][q] * c[q];
        c[row] = s / A[row][row];
    }
    if (N == 1) c[1] = 0.0;  // exact: the identity term vanishes for the first-order kernel
}

template <typename T>
void fill_consts(yy_filter* f, Consts<T>* k, const double* halfwidth) {
    const yy_config& c = f->cfg;
    k->n = c.n;
    k->n_pad = f->n_pad;
    k->r = c.r;
    k->r_pad = f->r_pad;
    k->N = c.n_scales;
    k->model = c.model;
    k->model_a = (T)c.model_a;
    k->tc_prefix = c.screen_prefix > 0 ? c.screen_prefix : 0;
    // symmetric blocks need the long-row epilogue (r > 64)
    k->tc_sym = (c.precision == YY_PREC_BF16 && c.r > 64) ? 1 : 0;
    k->tc_split_len = 64;
    // Screen operands.  BF16: |dG| <= 2^-6 |u_i||u_s| (unit roundoff 2^-9 per operand, 4x
    // slack).  FP8 e4m3 of s u, s the largest power of two with s 8 max R <= 448 (a learned
    // box is at most 8 times wider): per product (2 2^-4 + 2^-8) |a b| = 0.129 |a b|, plus
    // at most 2^-9 for reduced-precision accumulation inside one instruction (bound 0.14), and
    // for subnormal codes an absolute error delta = 2^-10 / s per coordinate, which adds
    // 1.07 delta sqrt(K) (|a| + |b|) + K delta^2 to |dG| (K coordinates); the d^2 bound is
    // twice these, with 10 % slack.
    k->tc_fp8 = (c.precision == YY_PREC_BF16 && c.screen_type == YY_SCREEN_FP8) ? 1 : 0;
    k->tc_r8 = (int)((f->r_pad + 127) / 128 * 128);
    k->tc_s = 1.f;
    k->tc_g2 = -2.f;
    k->tc_eps = 0.015625f;
    k->tc_dabs = 0.f;
    k->tc_dabs2 = 0.f;
    if (k->tc_fp8) {
        double rmax = 0.0;
        for (int d = 0; d < c.r; ++d) rmax = fmax(rmax, halfwidth ? halfwidth[d] : c.R);
        double s = 1.0;
        while (s * 8.0 * rmax * 2.0 <= 448.0 && s < 1048576.0) s *= 2.0;
        while (s * 8.0 * rmax > 448.0 && s > 1.0 / 1048576.0) s *= 0.5;
        const double K = (double)k->tc_r8, delta = ldexp(1.0, -10) / s;
        k->tc_s = (float)s;
        k->tc_g2 = (float)(-2.0 / (s * s));
        k->tc_eps = 0.14f;
        k->tc_dabs = (float)(1.1 * 2.0 * 1.07 * delta * sqrt(K));
        k->tc_dabs2 = (float)(1.1 * 2.0 * K * delta * delta);
    }
    k->dt = (T)c.dt;
    double log_vol = 0.0;
    for (int d = 0; d < c.r; ++d) log_vol += log(2.0 * (halfwidth ? halfwidth[d] : c.R));
    f->log_wq = log_vol - log((double)c.n);
    double Cj[kMaxScales];
    double cref = -INFINITY;
    for (int j = 0; j < c.n_scales; ++j) {
        const double tau = c.dt / ldexp(1.0, j);
        Cj[j] = -0.5 * c.r * log(2.0 * M_PI * tau) + f->log_wq;
        cref = fmax(cref, Cj[j]);
        k->tau[j] = (T)tau;
        k->inv2tau[j] = (T)(0.5 / tau);
    }
    for (int j = 0; j < c.n_scales; ++j) k->cj_off[j] = (T)(Cj[j] - cref);
    for (int j = c.n_scales; j < kMaxScales; ++j) { k->tau[j] = T(0); k->inv2tau[j] = T(0); k->cj_off[j] = T(0); }
    for (int j = 0; j <= kMaxScales; ++j) { k->logabs_c[j] = T(0); k->sign_c[j] = T(0); }
    for (int j = 0; j <= c.n_scales; ++j) {
        const double cj = f->coef[j];
        k->sign_c[j] = (cj > 0.0) ? T(1) : (cj < 0.0 ? T(-1) : T(0));
        k->logabs_c[j] = (cj != 0.0) ? (T)log(fabs(cj)) : T(0);
    }
    k->c_ref = cref;
    f->c_ref = cref;
    k->wait_ns = f->wait_ns;
    k->row0 = f->row0;
    k->row1 = f->row1;
    k->noise = c.noise;
    k->noise_u_zero = c.noise_u_zero;
    k->nz_u = (T)c.noise_u;
    k->nz_uk = (T)c.noise_u_kappa;
    k->nz_v = (T)c.noise_v;
    k->nz_vk = (T)c.noise_v_kappa;
}

yy_status cuda_status(cudaError_t e) { return e == cudaSuccess ? YY_OK : YY_ERR_CUDA; }

__global__ void k_set_stats(DevStats* st, double lognorm, long long step) {
    st->lognorm = lognorm;
    st->step = step;
    st->op_stale = 1;   // the centre may have moved
}

__global__ void k_init_cref(DevStats* st, double c_ref) {
    st->c_ref = c_ref;
    st->op_stale = 1;   // a new node set
}

// The first `count` primes (trial division by the primes found so far).
std::vector<uint32_t> first_primes_host(int count) {
    std::vector<uint32_t> ps;
    for (uint32_t c = 2; (int)ps.size() < count; ++c) {
        bool prime = true;
        for (uint32_t q : ps) {
            if (q * q > c) break;
            if (c % q == 0) { prime = false; break; }
        }
        if (prime) ps.push_back(c);
    }
    return ps;
}

uint32_t smallest_prime_at_least_host(uint32_t m) {
    for (uint32_t c = m < 2 ? 2 : m;; ++c) {
        bool prime = true;
        for (uint32_t q = 2; q * q <= c; ++q)
            if (c % q == 0) { prime = false; break; }
        if (prime) return c;
    }
}

// node_kind: YY_NODES_SOBOL (h_poly, h_scr: the Sobol parameters) or Halton / Faure.
template <typename T>
yy_status do_init_nodes(yy_filter* f, Bufs<T>& b, Consts<T>& k, const uint32_t* h_poly,
                        const uint32_t* h_scr, const double* h_center, const double* h_half,
                        int node_kind = YY_NODES_SOBOL) {
    const yy_config& c = f->cfg;
    const int W = YY_SOBOL_POLY_WORDS + YY_SOBOL_SCRAMBLE_WORDS;
    uint32_t* staging = (uint32_t*)calloc((size_t)c.r * W, sizeof(uint32_t));
    double* cen = (double*)calloc(f->r_pad, sizeof(double));
    double* half = (double*)calloc(f->r_pad, sizeof(double));
    if (!staging || !cen || !half) { free(staging); free(cen); free(half); return YY_ERR_ARG; }
    const std::vector<uint32_t> primes = node_kind == YY_NODES_HALTON ? first_primes_host(c.r) : std::vector<uint32_t>();
    for (int d = 0; d < c.r; ++d) {
        if (node_kind == YY_NODES_SOBOL) {
            memcpy(staging + (size_t)d * W, h_poly + (size_t)d * YY_SOBOL_POLY_WORDS,
                   sizeof(uint32_t) * YY_SOBOL_POLY_WORDS);
            uint32_t* L = staging + (size_t)d * W + YY_SOBOL_POLY_WORDS;
            if (h_scr) {
                memcpy(L, h_scr + (size_t)d * YY_SOBOL_SCRAMBLE_WORDS, sizeof(uint32_t) * YY_SOBOL_SCRAMBLE_WORDS);
            } else {
                for (int q = 1; q <= 32; ++q) L[q - 1] = 1u << (32 - q);
                L[32] = 0u;
            }
        } else if (node_kind == YY_NODES_HALTON) {
            staging[d] = primes[d];   // the staging area holds the bases
        }
        cen[d] = h_center[d];
        half[d] = h_half ? h_half[d] : c.R;
    }
    fill_consts<T>(f, &k, half);
    cudaStream_t s = f->stream;
    cudaError_t e = cudaMemcpyAsync(b.params, staging, sizeof(uint32_t) * (size_t)c.r * W, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.centre, cen, sizeof(double) * f->r_pad, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.halfwidth, half, sizeof(double) * f->r_pad, cudaMemcpyHostToDevice, s);
    // pageable copies are staged before return, but keep the host buffers until the stream drains
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    free(staging); free(cen); free(half);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    if (node_kind == YY_NODES_SOBOL) {
        if ((e = launch_sobol_dirs<T>(b.params, b.dirs, c.r, s)) != cudaSuccess) return YY_ERR_CUDA;
        if ((e = launch_sobol_points(b.dirs, c.r, f->r_pad, 0, c.n, b.u, nullptr, b.halfwidth, s)) != cudaSuccess)
            return YY_ERR_CUDA;
    } else {
        const uint32_t pf = smallest_prime_at_least_host((uint32_t)c.r);
        if ((e = launch_lds_points(node_kind, b.params, pf, c.r, f->r_pad, c.n, b.u, b.halfwidth, s)) != cudaSuccess)
            return YY_ERR_CUDA;
    }
    f->node_kind = node_kind;
    if ((e = launch_prep<T>(k, b, true, true, c.prior_mean, c.prior_var, s)) != cudaSuccess) return YY_ERR_CUDA;
    int l = 0;
    if ((e = launch_normalise_only<T>(k, b, s, &l)) != cudaSuccess) return YY_ERR_CUDA;
    k_set_stats<<<1, 1, 0, s>>>(b.stats, 0.0, 0);
    k_init_cref<<<1, 1, 0, s>>>(b.stats, f->c_ref);
    f->launches += 6 + l;
    if (f->cfg.precision == YY_PREC_BF16) {
        const yy_status st = build_tc_schedule(f);
        if (st != YY_OK) return st;
    }
    f->nodes_ready = true;
    f->predicted = false;
    return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" {

size_t yy_workspace_bytes(const yy_config* cfg) {
    if (!cfg_valid(cfg)) return 0;
    if (cfg->precision == YY_PREC_FP64) return carve<double>(cfg, nullptr, nullptr);
    return carve<float>(cfg, nullptr, nullptr);
}

yy_status yy_create(const yy_config* cfg, void* d_workspace, size_t bytes, void* stream,
                    yy_filter** out) {
    if (!out) return YY_ERR_ARG;
    *out = nullptr;
    if (!cfg_valid(cfg)) return YY_ERR_ARG;
    if (!cfg_supported(cfg)) return YY_ERR_UNSUPPORTED;
    const size_t need = yy_workspace_bytes(cfg);
    if (!d_workspace || ((uintptr_t)d_workspace & 255u) || bytes < need) return YY_ERR_WORKSPACE;
    yy_filter* f = new (std::nothrow) yy_filter();
    if (!f) return YY_ERR_ARG;
    f->cfg = *cfg;
    f->r_pad = (int)round_up(cfg->r, kColAlign);
    f->n_pad = round_up(cfg->n, kRowAlign);
    f->stream = (cudaStream_t)stream;
    f->ws = (char*)d_workspace;
    f->ws_bytes = bytes;
    f->fp64 = (cfg->precision == YY_PREC_FP64);
    f->wait_ns = kDefaultWaitNs;
    f->pair_ok = false;
    f->kf.wait_ns = f->kd.wait_ns = kDefaultWaitNs;
    f->row0 = 0;
    f->row1 = cfg->n;
    f->shard_rank = 0;
    f->shard_count = 1;
    f->use_op = (cfg->materialise == 2);
    multiscale_coefficients(cfg->n_scales, f->coef);
    if (f->fp64) carve<double>(cfg, f->ws, &f->bd);
    else carve<float>(cfg, f->ws, &f->bf);
    cudaError_t e = cudaSuccess;
    if (cfg->precision == YY_PREC_BF16) e = prepare_ksum_tc();
    if (e == cudaSuccess && cfg->materialise && !f->fp64) e = prepare_op_apply();
    if (e == cudaSuccess) e = cudaMemsetAsync(d_workspace, 0, need, f->stream);
    if (e != cudaSuccess) { delete f; return YY_ERR_CUDA; }
    *out = f;
    return YY_OK;
}

yy_status yy_destroy(yy_filter* f) {
    if (f) {
        if (f->gexec) cudaGraphExecDestroy(f->gexec);
        if (f->graph) cudaGraphDestroy(f->graph);
    }
    delete f;
    return YY_OK;
}

yy_status yy_init_nodes(yy_filter* f, const uint32_t* h_poly, const uint32_t* h_scramble,
                        const double* h_center, const double* h_halfwidth) {
    if (!f || !h_poly || !h_center) return YY_ERR_ARG;
    for (int d = 0; d < f->cfg.r; ++d) {
        const uint32_t s = h_poly[(size_t)d * YY_SOBOL_POLY_WORDS];
        if (s > YY_SOBOL_POLY_WORDS - 2) return YY_ERR_ARG;
        if (h_halfwidth && !(h_halfwidth[d] > 0.0)) return YY_ERR_ARG;
        if (!isfinite(h_center[d])) return YY_ERR_ARG;
    }
    if (f->fp64) return do_init_nodes<double>(f, f->bd, f->kd, h_poly, h_scramble, h_center, h_halfwidth);
    return do_init_nodes<float>(f, f->bf, f->kf, h_poly, h_scramble, h_center, h_halfwidth);
}

yy_status yy_init_nodes_lds(yy_filter* f, int32_t kind, const double* h_center, const double* h_halfwidth) {
    if (!f || !h_center || (kind != YY_NODES_HALTON && kind != YY_NODES_FAURE)) return YY_ERR_ARG;
    if (f->mlp && f->cfg.restart_rule == YY_RESTART_LEARNED) return YY_ERR_UNSUPPORTED;
    for (int d = 0; d < f->cfg.r; ++d) {
        if (h_halfwidth && !(h_halfwidth[d] > 0.0)) return YY_ERR_ARG;
        if (!isfinite(h_center[d])) return YY_ERR_ARG;
    }
    if (f->fp64) return do_init_nodes<double>(f, f->bd, f->kd, nullptr, nullptr, h_center, h_halfwidth, kind);
    return do_init_nodes<float>(f, f->bf, f->kf, nullptr, nullptr, h_center, h_halfwidth, kind);
}

yy_status yy_sobol_bits(yy_filter* f, uint32_t* d_bits, int64_t first, int64_t count) {
    if (!f || !d_bits || first < 0 || count < 0) return YY_ERR_ARG;
    if (!f->nodes_ready) return YY_ERR_STATE;
    if (f->node_kind != YY_NODES_SOBOL) return YY_ERR_UNSUPPORTED;
    const uint32_t* dirs = f->fp64 ? f->bd.dirs : f->bf.dirs;
    f->launches += 1;
    return cuda_status(launch_sobol_points(dirs, f->cfg.r, f->r_pad, first, count, nullptr, d_bits,
                                           nullptr, f->stream));
}

yy_status yy_predict(yy_filter* f) {
    if (!f) return YY_ERR_ARG;
    if (!f->nodes_ready) return YY_ERR_STATE;
    cudaError_t e;
    if (f->fp64) {
        e = cudaMemsetAsync(&f->bd.stats->clamps, 0, sizeof(unsigned), f->stream);
        int l = 0;
        if (e == cudaSuccess) e = launch_ksum_simt<double>(f->kd, f->bd, f->stream, &l);
        f->launches += l;
    } else if (f->use_op) {
        // materialised schedule: rebuild on the device if the node set moved, then apply
        e = cudaMemsetAsync(&f->bf.stats->clamps, 0, sizeof(unsigned), f->stream);
        if (e == cudaSuccess) e = launch_op_build(f->kf, f->bf, false, f->stream);
        if (e == cudaSuccess) e = launch_op_apply(f->kf, f->bf, f->stream);
        f->launches += 3;   // build (returns at once unless the node set moved), source terms, apply
    } else if (f->cfg.precision == YY_PREC_FP32 || f->route_plain) {
        e = cudaMemsetAsync(&f->bf.stats->clamps, 0, sizeof(unsigned), f->stream);
        int l = 0;
        if (e == cudaSuccess) e = launch_ksum_simt<float>(f->kf, f->bf, f->stream, &l);
        f->launches += l;
    } else if (f->cfg.precision == YY_PREC_FP32_SCREEN) {
        // first pass over 64 k coordinates: k = screen_prefix, else half of the 64-chunks
        const int nk = f->r_pad / kColAlign;
        const int k1 = kColAlign * (f->cfg.screen_prefix > 0 ? f->cfg.screen_prefix : (nk + 1) / 2);
        e = cudaMemsetAsync(&f->bf.stats->clamps, 0, sizeof(unsigned), f->stream);
        if (e == cudaSuccess) e = launch_ksum_scr32(f->kf, f->bf, k1, f->stream);
        f->launches += 2;
    } else {
        e = cudaMemsetAsync(&f->bf.stats->clamps, 0, sizeof(unsigned), f->stream);
        int l = 0;
        if (e == cudaSuccess) e = launch_ksum_tc(f->kf, f->bf, f->stream, &l);
        f->launches += l;
        if (e == cudaErrorNotSupported) return YY_ERR_UNSUPPORTED;
    }
    if (e != cudaSuccess) return YY_ERR_CUDA;
    f->predicted = true;
    return YY_OK;
}

yy_status yy_update(yy_filter* f, const double* d_dy) {
    if (!f || !d_dy) return YY_ERR_ARG;
    if (!f->nodes_ready || !f->predicted) return YY_ERR_STATE;
    if (f->shard_count > 1) return YY_ERR_STATE;   // a shard updates with yy_update_shard
    int l = 0;
    cudaError_t e = f->fp64
        ? launch_update<double>(f->kd, f->bd, d_dy, f->cfg.restart_interval, f->cfg.ess_frac, f->stream, &l)
        : launch_update<float>(f->kf, f->bf, d_dy, f->cfg.restart_interval, f->cfg.ess_frac, f->stream, &l);
    f->launches += l;
    if (e != cudaSuccess) return YY_ERR_CUDA;
    f->predicted = false;
    return YY_OK;
}

static yy_status status_from_word(unsigned w) {
    if (w & kStatusTimeout) return YY_ERR_TIMEOUT;
    if (w & kStatusDegenerate) return YY_ERR_DEGENERATE;
    if (w & kStatusNonFinite) return YY_ERR_NONFINITE;
    return YY_OK;
}

yy_status yy_estimate(yy_filter* f, double* h_mean, double* h_var, double* h_ess, double* h_lognorm) {
    if (!f) return YY_ERR_ARG;
    if (!f->nodes_ready) return YY_ERR_STATE;
    DevStats* st = f->fp64 ? f->bd.stats : f->bf.stats;
    double* mean = f->fp64 ? f->bd.mean : f->bf.mean;
    double* var = f->fp64 ? f->bd.var : f->bf.var;
    DevStats hs;
    cudaError_t e = cudaMemcpyAsync(&hs, st, sizeof(DevStats), cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess && h_mean) e = cudaMemcpyAsync(h_mean, mean, sizeof(double) * f->cfg.r, cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess && h_var) e = cudaMemcpyAsync(h_var, var, sizeof(double) * f->cfg.r, cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    if (h_ess) *h_ess = hs.ess;
    if (h_lognorm) *h_lognorm = hs.lognorm;
    return status_from_word(hs.status);
}

yy_status yy_restart(yy_filter* f, int32_t mode, int32_t* h_did_restart) {
    if (!f) return YY_ERR_ARG;
    if (mode != YY_RESTART_AUTO && mode != YY_RESTART_FORCE && mode != YY_RESTART_NEVER) return YY_ERR_ARG;
    if (!f->nodes_ready || f->predicted || f->shard_updated) return YY_ERR_STATE;
    int l = 0;
    yy_mlp* net = (f->cfg.restart_rule == YY_RESTART_LEARNED) ? f->mlp : nullptr;
    cudaError_t e = f->fp64
        ? launch_restart<double>(f->kd, f->bd, mode, f->cfg.restart_init, f->cfg.R, net, f->stream, &l)
        : launch_restart<float>(f->kf, f->bf, mode, f->cfg.restart_init, f->cfg.R, net, f->stream, &l);
    f->launches += l;
    if (e != cudaSuccess) return YY_ERR_CUDA;
    if (h_did_restart) {
        DevStats* st = f->fp64 ? f->bd.stats : f->bf.stats;
        if (mode == YY_RESTART_NEVER) {
            int flag = 0;
            e = cudaMemcpyAsync(&flag, &st->restart_flag, sizeof(int), cudaMemcpyDeviceToHost, f->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
            *h_did_restart = flag;
        } else {
            int did = 0;
            e = cudaMemcpyAsync(&did, &st->last_restarted, sizeof(int), cudaMemcpyDeviceToHost, f->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
            *h_did_restart = did;
        }
        if (e != cudaSuccess) return YY_ERR_CUDA;
    }
    return YY_OK;
}

yy_status yy_run_steps(yy_filter* f, const double* d_dy_all, int64_t K, double* d_hist) {
    if (!f || !d_dy_all || K < 0) return YY_ERR_ARG;
    if (!f->nodes_ready || f->predicted || f->shard_count > 1) return YY_ERR_STATE;
    const int r = f->cfg.r;
    for (int64_t k = 0; k < K; ++k) {
        yy_status st = yy_predict(f);
        if (st != YY_OK) return st;
        if ((st = yy_update(f, d_dy_all + (size_t)k * f->cfg.m)) != YY_OK) return st;
        if (d_hist) {
            double* row = d_hist + (size_t)k * (2 * r + 4);
            cudaError_t e = f->fp64 ? launch_record<double>(f->kd, f->bd, row, f->stream)
                                    : launch_record<float>(f->kf, f->bf, row, f->stream);
            if (e != cudaSuccess) return YY_ERR_CUDA;
            f->launches += 1;
        }
        if ((st = yy_restart(f, YY_RESTART_AUTO, nullptr)) != YY_OK) return st;
    }
    return YY_OK;
}

yy_status yy_graph_capture(yy_filter* f, const double* d_dy_all, int64_t K, double* d_hist) {
    if (!f || !d_dy_all || K < 1) return YY_ERR_ARG;
    if (!f->stream) return YY_ERR_STATE;
    if (!f->nodes_ready || f->predicted) return YY_ERR_STATE;
    if (f->gexec) { cudaGraphExecDestroy(f->gexec); f->gexec = nullptr; }
    if (f->graph) { cudaGraphDestroy(f->graph); f->graph = nullptr; }
    const long long l0 = f->launches;
    cudaError_t e = cudaStreamBeginCapture(f->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    const yy_status st = yy_run_steps(f, d_dy_all, K, d_hist);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(f->stream, &g);
    f->graph_kernels = f->launches - l0;
    f->launches = l0;   // capture launches nothing
    f->predicted = false;
    if (st != YY_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return YY_ERR_CUDA;
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(g); return YY_ERR_CUDA; }
    f->graph = g;
    f->gexec = ex;
    return YY_OK;
}

yy_status yy_graph_launch(yy_filter* f) {
    if (!f) return YY_ERR_ARG;
    if (!f->gexec) return YY_ERR_STATE;
    f->launches += f->graph_kernels;
    return cuda_status(cudaGraphLaunch(f->gexec, f->stream));
}

int64_t yy_graph_kernel_count(const yy_filter* f) { return (f && f->gexec) ? f->graph_kernels : 0; }

yy_status yy_get_nodes(yy_filter* f, float* h_u, uint8_t* h_mask) {
    if (!f) return YY_ERR_ARG;
    if (!f->nodes_ready) return YY_ERR_STATE;
    const float* u = f->fp64 ? f->bd.u : f->bf.u;
    const uint8_t* mk = f->fp64 ? f->bd.mask : f->bf.mask;
    cudaError_t e = cudaSuccess;
    if (h_u)
        e = cudaMemcpy2DAsync(h_u, sizeof(float) * f->cfg.r, u, sizeof(float) * f->r_pad,
                              sizeof(float) * f->cfg.r, (size_t)f->cfg.n, cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess && h_mask) e = cudaMemcpyAsync(h_mask, mk, (size_t)f->cfg.n, cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    return cuda_status(e);
}

yy_status yy_get_log_weights(yy_filter* f, void* h_logw, double* h_offset) {
    if (!f || !h_logw) return YY_ERR_ARG;
    if (!f->nodes_ready) return YY_ERR_STATE;
    const size_t es = f->fp64 ? sizeof(double) : sizeof(float);
    const void* src = f->predicted ? (f->fp64 ? (void*)f->bd.logw_pred : (void*)f->bf.logw_pred)
                                   : (f->fp64 ? (void*)f->bd.logw : (void*)f->bf.logw);
    DevStats* st = f->fp64 ? f->bd.stats : f->bf.stats;
    double cref = 0.0;
    cudaError_t e = cudaMemcpyAsync(h_logw, src, es * (size_t)f->cfg.n, cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cref, &st->c_ref, sizeof(double), cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (h_offset) *h_offset = f->predicted ? cref : 0.0;
    return cuda_status(e);
}

yy_status yy_set_state(yy_filter* f, const double* h_center, const void* h_logw, double lognorm,
                       int64_t step) {
    if (!f || !h_center || !h_logw || step < 0) return YY_ERR_ARG;
    if (!f->nodes_ready) return YY_ERR_STATE;
    for (int d = 0; d < f->cfg.r; ++d)
        if (!isfinite(h_center[d])) return YY_ERR_ARG;
    const size_t es = f->fp64 ? sizeof(double) : sizeof(float);
    double* cen = f->fp64 ? f->bd.centre : f->bf.centre;
    void* lw = f->fp64 ? (void*)f->bd.logw : (void*)f->bf.logw;
    DevStats* st = f->fp64 ? f->bd.stats : f->bf.stats;
    cudaError_t e = cudaMemcpyAsync(cen, h_center, sizeof(double) * f->cfg.r, cudaMemcpyHostToDevice, f->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lw, h_logw, es * (size_t)f->cfg.n, cudaMemcpyHostToDevice, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    k_set_stats<<<1, 1, 0, f->stream>>>(st, lognorm, step);
    e = f->fp64 ? launch_prep<double>(f->kd, f->bd, false, false, 0.0, 1.0, f->stream)
                : launch_prep<float>(f->kf, f->bf, false, false, 0.0, 1.0, f->stream);
    f->launches += 3;
    f->predicted = false;
    return cuda_status(e);
}

yy_status yy_set_restart_mlp(yy_filter* f, yy_mlp* net) {
    if (!f) return YY_ERR_ARG;
    if (net && f->fp64) return YY_ERR_UNSUPPORTED;
    if (net && f->nodes_ready && f->node_kind != YY_NODES_SOBOL) return YY_ERR_UNSUPPORTED;
    f->mlp = net;
    return YY_OK;
}

yy_status yy_get_box(yy_filter* f, double* h_center, double* h_halfwidth) {
    if (!f) return YY_ERR_ARG;
    if (!f->nodes_ready) return YY_ERR_STATE;
    const double* cen = f->fp64 ? f->bd.centre : f->bf.centre;
    const double* half = f->fp64 ? f->bd.halfwidth : f->bf.halfwidth;
    cudaError_t e = cudaSuccess;
    if (h_center) e = cudaMemcpyAsync(h_center, cen, sizeof(double) * f->cfg.r, cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess && h_halfwidth)
        e = cudaMemcpyAsync(h_halfwidth, half, sizeof(double) * f->cfg.r, cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    return cuda_status(e);
}

yy_status yy_get_state(yy_filter* f, double* h_center, double* h_lognorm, int64_t* h_step) {
    if (!f) return YY_ERR_ARG;
    if (!f->nodes_ready) return YY_ERR_STATE;
    double* cen = f->fp64 ? f->bd.centre : f->bf.centre;
    DevStats* st = f->fp64 ? f->bd.stats : f->bf.stats;
    DevStats hs;
    cudaError_t e = cudaMemcpyAsync(&hs, st, sizeof(DevStats), cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess && h_center)
        e = cudaMemcpyAsync(h_center, cen, sizeof(double) * f->cfg.r, cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    if (h_lognorm) *h_lognorm = hs.lognorm;
    if (h_step) *h_step = hs.step;
    return YY_OK;
}

yy_status yy_get_clamps(yy_filter* f, int64_t* h_clamps) {
    if (!f || !h_clamps) return YY_ERR_ARG;
    DevStats* st = f->fp64 ? f->bd.stats : f->bf.stats;
    DevStats hs;
    cudaError_t e = cudaMemcpyAsync(&hs, st, sizeof(DevStats), cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    *h_clamps = hs.clamps;
    return YY_OK;
}

int64_t yy_launch_count(const yy_filter* f) { return f ? f->launches : 0; }

yy_status yy_tune_materialise(yy_filter* f, int32_t predicts_per_build, int32_t reps, double* h_ms,
                               int32_t* h_choice) {
    if (!f || predicts_per_build < 1 || reps < 1) return YY_ERR_ARG;
    if (f->cfg.materialise == 0 || f->fp64 || !f->bf.op) return YY_ERR_UNSUPPORTED;
    if (!f->nodes_ready || f->predicted || f->shard_updated) return YY_ERR_STATE;
    cudaEvent_t ev[6];
    for (auto& x : ev)
        if (cudaEventCreate(&x) != cudaSuccess) return YY_ERR_CUDA;
    const bool keep = f->use_op;
    cudaError_t e = cudaSuccess;
    // recomputed prediction
    f->use_op = false;
    cudaEventRecord(ev[0], f->stream);
    for (int q = 0; q < reps && e == cudaSuccess; ++q) e = (yy_predict(f) == YY_OK) ? cudaSuccess : cudaErrorUnknown;
    cudaEventRecord(ev[1], f->stream);
    // build (forced) and apply
    for (int q = 0; q < reps && e == cudaSuccess; ++q) e = launch_op_build(f->kf, f->bf, true, f->stream);
    cudaEventRecord(ev[2], f->stream);
    for (int q = 0; q < reps && e == cudaSuccess; ++q) e = launch_op_apply(f->kf, f->bf, f->stream);
    cudaEventRecord(ev[3], f->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
    float t_re = 0.f, t_build = 0.f, t_apply = 0.f;
    if (e == cudaSuccess) {
        cudaEventElapsedTime(&t_re, ev[0], ev[1]);
        cudaEventElapsedTime(&t_build, ev[1], ev[2]);
        cudaEventElapsedTime(&t_apply, ev[2], ev[3]);
    }
    for (auto& x : ev) cudaEventDestroy(x);
    f->launches += (int64_t)reps * 2;
    f->predicted = false;   // the timing predictions leave the weights as they were
    if (e != cudaSuccess) { f->use_op = keep; return YY_ERR_CUDA; }
    const double re = t_re / reps, bu = t_build / reps, ap = t_apply / reps;
    f->use_op = (f->cfg.materialise == 2) || (bu + predicts_per_build * ap < predicts_per_build * re);
    if (h_ms) { h_ms[0] = re; h_ms[1] = bu; h_ms[2] = ap; }
    if (h_choice) *h_choice = f->use_op ? 1 : 0;
    return YY_OK;
}

// Routes a BF16 filter's predictions to the plain float32 form (or back).  The plain form
// reads the stored drift f; a filter that did not store it gets it for its current nodes
// from the preparation pass, and stores it from then on.  Back on the screen, the drift is
// recomputed from u inside the screen again (except for the model whose drift is always
// stored).
static yy_status route_to(yy_filter* f, bool plain) {
    const int screen_store_f = (f->cfg.model == YY_MODEL_PAPER_E1) ? 1 : 0;
    cudaError_t e = cudaSuccess;
    if (plain && !f->bf.store_f) {
        f->bf.store_f = 1;
        if (f->nodes_ready) {
            e = launch_prep<float>(f->kf, f->bf, false, false, 0.0, 1.0, f->stream);
            f->launches += 1;
        }
    } else if (!plain) {
        f->bf.store_f = screen_store_f;
    }
    f->route_plain = plain;
    return cuda_status(e);
}

yy_status yy_set_route(yy_filter* f, int32_t plain) {
    if (!f || (plain != 0 && plain != 1)) return YY_ERR_ARG;
    if (f->cfg.precision != YY_PREC_BF16) return YY_ERR_UNSUPPORTED;
    if (f->predicted || f->shard_updated) return YY_ERR_STATE;
    return route_to(f, plain == 1);
}

yy_status yy_tune_route(yy_filter* f, int32_t reps, double* h_ms, int32_t* h_route) {
    if (!f || reps < 1) return YY_ERR_ARG;
    if (f->cfg.precision != YY_PREC_BF16) return YY_ERR_UNSUPPORTED;
    if (!f->nodes_ready || f->predicted || f->shard_updated) return YY_ERR_STATE;
    const bool keep_op = f->use_op;
    f->use_op = false;   // the two forms compared are the recomputing ones
    cudaEvent_t ev[4];
    for (auto& x : ev)
        if (cudaEventCreate(&x) != cudaSuccess) { f->use_op = keep_op; return YY_ERR_CUDA; }
    yy_status st = route_to(f, true);   // f of the current nodes, stored
    auto predicts = [&](int m) {
        for (int q = 0; q < m && st == YY_OK; ++q) st = yy_predict(f);
    };
    predicts(1);
    cudaEventRecord(ev[0], f->stream);
    predicts(reps);
    cudaEventRecord(ev[1], f->stream);
    // the screen as it runs when chosen (drift recomputed inside it); f stays valid in
    // memory, since the timing leaves the nodes as they are
    f->bf.store_f = (f->cfg.model == YY_MODEL_PAPER_E1) ? 1 : 0;
    f->route_plain = false;
    predicts(1);
    cudaEventRecord(ev[2], f->stream);
    predicts(reps);
    cudaEventRecord(ev[3], f->stream);
    cudaError_t e = st == YY_OK ? cudaEventSynchronize(ev[3]) : cudaSuccess;
    float t_plain = 0.f, t_screen = 0.f;
    if (st == YY_OK && e == cudaSuccess) {
        cudaEventElapsedTime(&t_plain, ev[0], ev[1]);
        cudaEventElapsedTime(&t_screen, ev[2], ev[3]);
    }
    for (auto& x : ev) cudaEventDestroy(x);
    f->predicted = false;   // the timing predictions leave the weights as they were
    f->use_op = keep_op;
    if (st != YY_OK || e != cudaSuccess) {   // back on the screen, the default route
        route_to(f, false);
        return st != YY_OK ? st : YY_ERR_CUDA;
    }
    const bool plain = t_plain < t_screen;
    if (plain) {   // f is still that of the current nodes
        f->bf.store_f = 1;
        f->route_plain = true;
    }
    if (h_ms) { h_ms[0] = t_screen / reps; h_ms[1] = t_plain / reps; }
    if (h_route) *h_route = plain ? 1 : 0;
    return YY_OK;
}

yy_status yy_set_wait_limit(yy_filter* f, double seconds) {
    if (!f || !(seconds > 0.0) || seconds > 3600.0) return YY_ERR_ARG;
    unsigned long long ns = (unsigned long long)(seconds * 1e9);
    if (ns < 1) ns = 1;
    f->wait_ns = ns;
    f->kf.wait_ns = ns;
    f->kd.wait_ns = ns;
    return YY_OK;
}

yy_status yy_set_cta_pair(yy_filter* f, int32_t on, int32_t* h_pairs) {
    if (!f || (on != 0 && on != 1)) return YY_ERR_ARG;
    f->pair_ok = (on == 1);
    if (f->cfg.precision == YY_PREC_BF16 && f->nodes_ready) {
        const yy_status st = build_tc_schedule(f);
        if (st != YY_OK) return st;
    }
    if (h_pairs)
        *h_pairs = (f->cfg.precision == YY_PREC_BF16 && f->nodes_ready && f->bf.tc_pair) ? f->bf.tc_grid / 2 : 0;
    return YY_OK;
}

yy_status yy_get_counters(yy_filter* f, int64_t* h_clamps, int64_t* h_exact_pairs) {
    if (!f) return YY_ERR_ARG;
    DevStats* st = f->fp64 ? f->bd.stats : f->bf.stats;
    DevStats hs;
    cudaError_t e = cudaMemcpyAsync(&hs, st, sizeof(DevStats), cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    if (h_clamps) *h_clamps = hs.clamps;
    if (h_exact_pairs) *h_exact_pairs = (int64_t)hs.candidates;
    return YY_OK;
}

yy_status yy_get_screen(yy_filter* f, int32_t* h_last_prefix, int32_t* h_next_prefix, int64_t* h_tiles,
                        int64_t* h_rescreened) {
    if (!f) return YY_ERR_ARG;
    if (f->cfg.precision != YY_PREC_BF16) return YY_ERR_UNSUPPORTED;
    DevStats hs;
    cudaError_t e = cudaMemcpyAsync(&hs, f->bf.stats, sizeof(DevStats), cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return YY_ERR_CUDA;
    const int nk = f->kf.tc_fp8 ? f->kf.tc_r8 / 128 : (int)(f->r_pad / kColAlign);
    int v = f->cfg.screen_prefix > 0 ? f->cfg.screen_prefix : hs.tc_nk1;
    if (v <= 0) v = (nk + 1) / 2;
    if (h_last_prefix) *h_last_prefix = hs.tc_last_nk1;
    if (h_next_prefix) *h_next_prefix = std::max(1, std::min(v, nk));
    if (h_tiles) *h_tiles = (int64_t)hs.tc_last_blk;
    if (h_rescreened) *h_rescreened = (int64_t)hs.tc_last_esc;
    return YY_OK;
}

const char* yy_status_str(yy_status s) {
    switch (s) {
        case YY_OK: return "YY_OK";
        case YY_ERR_ARG: return "YY_ERR_ARG: invalid argument";
        case YY_ERR_CUDA: return "YY_ERR_CUDA: CUDA runtime error";
        case YY_ERR_WORKSPACE: return "YY_ERR_WORKSPACE: workspace missing, misaligned or too small";
        case YY_ERR_NONFINITE: return "YY_ERR_NONFINITE: non-finite normaliser or estimate";
        case YY_ERR_DEGENERATE: return "YY_ERR_DEGENERATE: every log-weight is -inf";
        case YY_ERR_TIMEOUT: return "YY_ERR_TIMEOUT: a device-side wait gave up";
        case YY_ERR_STATE: return "YY_ERR_STATE: call out of order";
        case YY_ERR_UNSUPPORTED: return "YY_ERR_UNSUPPORTED: configuration not supported";
    }
    return "unknown yy_status";
}

}  // extern "C"
