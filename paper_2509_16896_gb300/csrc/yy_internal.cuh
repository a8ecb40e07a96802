// Internal declarations of libyy (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <math.h>

#include "yy.h"

struct yy_mlp;

namespace yy {

constexpr int kMaxScales = YY_MAX_SCALES;
constexpr int kRowAlign = 256;       // node rows are padded to a multiple of this
constexpr int kColAlign = 64;        // coordinates per row are padded to a multiple of this
constexpr int kNumPartBlocks = 304;  // blocks of the reduction passes (2 per SM)
constexpr int kSimtMaxSplit = 8;     // source ranges per target block of the plain form

// Device status word bits (sticky until the handle is recreated).
constexpr uint32_t kStatusNonFinite = 1u << 0;
constexpr uint32_t kStatusDegenerate = 1u << 1;
constexpr uint32_t kStatusTimeout = 1u << 2;

// Device-side per-filter scalars.
struct DevStats {
    double lam_rel;      // log-sum-exp of the unnormalised log-weights, relative to offsets
    double lam;          // Lambda_k (absolute)
    double lognorm;      // Z_k
    double lam_c;        // Ito-corrected log-likelihood at the box centre
    double ess;
    double wsum, wsq;    // sum of normalised weights and of their squares
    long long step;      // k
    int restart_flag;    // test result of the last update (or forced)
    int restarts;        // restarts so far
    unsigned int status; // kStatus* bits
    unsigned int clamps; // non-positive combinations in the last predict
    unsigned long long candidates;  // exact pair evaluations in the last BF16 predict
    int last_restarted;  // 1 if the last yy_restart call re-centred the box
    int scale_changed;   // 1 while a restart re-maps the nodes to new half-widths
    double c_ref;        // offset of the predicted log-weights (moves with the box volume)
    int part_count;      // entries of part_list
    // tensor-core screen: stages (64 BF16 or 128 e4m3 coordinates) of the first pass and its controller
    int tc_nk1;          // 0 = not chosen yet
    int tc_streak;       // consecutive clean predictions at the current length
    int tc_from;         // first-pass length of the prediction before the last one
    int tc_hold[YY_MAX_DIM / 64 + 1];     // predictions a length is still held off
    unsigned long long tc_blk;   // tiles screened by the last prediction
    unsigned long long tc_esc;   // of which rescreened with all coordinates
    unsigned long long tc_last_blk, tc_last_esc;   // the same, kept for the host
    int tc_last_nk1;             // first-pass chunks the last prediction used
    unsigned int tc_done;        // CTAs of the running prediction launch that finished
    float scr_lmax;              // screened float32 form: largest live source log-weight
    int op_stale;                // the materialised operator must be rebuilt (nodes moved)
};

// Constants of one filter handed to kernels by value.
template <typename T>
struct Consts {
    long long n, n_pad;
    int r, r_pad;
    int N;
    int model;           // yy_model
    T model_a;
    T dt;
    T tau[kMaxScales];
    T inv2tau[kMaxScales];   // 1 / (2 tau_j)
    T cj_off[kMaxScales];    // C_j - C_ref, C_j = -(r/2) log(2 pi tau_j) + log w_q
    int tc_prefix;           // fixed first-pass stages of the tensor-core screen (0 = adaptive)
    int tc_sym;              // screen over the upper block triangle, both directions per block
    int tc_split_len;        // symmetric screen: source tiles per work item (set with the work list)
    int tc_fp8;              // screen operands FP8 e4m3 (else BF16)
    int tc_r8;               // FP8: coordinates per row of the e4m3 copy (multiple of 128)
    float tc_s;              // FP8: power-of-two scale of the coordinates in the e4m3 copy
    float tc_g2;             // factor turning the accumulator into -2 G (-2, or -2 / s^2)
    float tc_eps;            // relative error bound of G per |u_i||u_s|
    float tc_dabs;           // FP8: absolute error term per (|u_i| + |u_s|) (subnormal codes)
    float tc_dabs2;          // FP8: constant error term
    T logabs_c[kMaxScales + 1];
    T sign_c[kMaxScales + 1];  // 0 for a zero coefficient
    double c_ref;
    unsigned long long wait_ns;  // limit of the prediction kernel's bounded waits (yy_set_wait_limit)
    long long row0, row1;        // target rows this handle predicts and updates: [0, n), or its
                                 // shard's equal chunk when the rows are split across devices
    int noise;                   // yy_noise
    int noise_u_zero;            // DIAG: coordinates without state noise
    T nz_u, nz_uk, nz_v, nz_vk;  // DIAG: U_d = nz_u (1 + nz_uk sin^2 x_d), V_d = nz_v (1 + nz_vk sin^2 x_d)
};

// Pointers into the caller's workspace.
template <typename T>
struct Bufs {
    float* u;             // [n_pad][r_pad] box coordinates
    T* f;                 // [n_pad][r_pad] drift at x = c + u
    __nv_bfloat16* ubf;   // [n_pad][r_pad] bf16 copy of u (BF16 precision only)
    T* divf;              // [n_pad]
    T* nu;                // [n_pad] |u_i|^2
    T* nf;                // [n_pad] |f_i|^2
    uint8_t* mask;        // [n_pad] Dirichlet boundary
    int store_f;          // f is written by the preparation pass (the BF16 screen of a single
                          // filter recomputes f of its few exact pairs instead)
    T* logw;              // [n_pad] current (normalised or unnormalised) log-weights
    T* logw_pred;         // [n_pad] predicted log-weights minus c_ref
    double* centre;       // [r_pad]
    double* halfwidth;    // [r_pad]
    uint32_t* dirs;       // [r][33] scrambled direction numbers + shift
    uint32_t* params;     // [r][16 + 33] staging of the Sobol parameters
    double* mean;         // [r_pad] x_hat
    double* var;          // [r_pad] v_hat
    T* obs_g;             // [r_pad] dy - dt h(c)
    T* obs_c;             // [r_pad] centre in T
    T* obs_l;             // [r_pad] noise coefficients: h(c) dy - dt/2 h(c)^2 per coordinate
    T* obs_ibc;           // [r_pad] noise coefficients: 1 / b_d(c)
    float* op;            // [N][n_pad][n_pad] materialised pair parts of log K_{tau_j} (materialise >= 1)
    float* op_lsrc;       // [n_pad] source terms of the materialised apply (log2 e ell_s, -inf if not live)
    T* minv;              // [n_pad][r_pad] noise coefficients: a(x)^+ (diagonal) at every node
    T* hld;               // [n_pad] noise coefficients: 1/2 log det_+ a(x)
    T* dimc;              // [5][r_pad] per-dimension constants of the preparation pass:
                          // centre head, tail, Gaussian restart 1 / (2 var), cos c, sin c
    double* next_centre;  // [r_pad] box of the restart in progress
    double* next_half;    // [r_pad]
    double* dy_last;      // [r_pad] observation increment of the last update
    double* part;         // reduction partials
    int* part_list;       // [kNumPartBlocks] moment partials with weight, in block order
    DevStats* stats;
    // tensor-core screen scratch (BF16 precision only)
    float* nu_chunk;      // [n_pad][r_pad / 64] |u_i|^2 per chunk of 64 coordinates (BF16 only)
    float* tc_q;          // [n_pad] |u_s|^2 of live sources, 3e38 for dead ones
    float* tc_q1;         // [n_pad] the same over the first-pass coordinates
    float* tc_q1t;        // [n_pad] first-pass |u_s|^2 of every node (as a target)
    float* tc_qmin;       // [n_pad / 32] smallest tc_q of each group of 32 sources
    float* tc_qmin1;      // [n_pad / 32] smallest tc_q1 of each group of 32 sources
    float* tc_qt;         // [n_pad] column-direction screen value of every node as a target:
                          // |u_c|^2 - (rho_c^2 + err_c) (+inf: no target, -inf: no bound)
    float* tc_qt1;        // [n_pad] the same over the first-pass coordinates
    float* tc_tile_rmax;  // [n_pad / 128] largest rho_c^2 + err_c of a chunk's targets (+inf: unbounded)
    float* tc_cinfo;      // [n_pad / 128][8] per chunk: lmax, numax, numax1, rmax, rmax1 (staged per tile)
    float* tc_tile_rmax1; // [n_pad / 128] the same over the first-pass coordinates
    unsigned long long* tc_xlse;   // [n_pad][kMaxScales] (max, sum) float pairs of the terms a
                                   // node receives as the column of a symmetric block
    float* tc_tile_lmax;  // [n_pad / 128] max live log-weight per chunk of 128 sources
    float* tc_tile_numax; // [n_pad / 128] max |u_s|^2 per chunk of 128 sources
    float* tc_tile_numax1;// [n_pad / 128] the same over the first-pass coordinates
    float* tc_part;       // [n_pad][8][4][2] partial (max, sum) of split work items
    T* simt_part;         // [n_pad][kSimtMaxSplit][kMaxScales][2] plain form: partial (max, sum)
                          // of each source range (filters with few target blocks only)
    int4* tc_items;       // single-filter work list (target tile, split, nsplit)
    int* tc_cta_start;    // [tc_grid + 1]
    int tc_grid;          // persistent CTAs of the single-filter prediction
    int tc_splits;        // source splits per target tile
    int tc_pair;          // 1: the work list is per 2-CTA cluster (items are pairs of target tiles)
};

// Device-side descriptor of one trajectory of a batch (kernels index it by blockIdx.y).
template <typename T>
struct Traj {
    Consts<T> k;
    Bufs<T> b;
    long long dy_off;      // offset of this trajectory's increments within a step row
    long long hist_off;    // offset of its record within a history row
    int restart_interval;
    double ess_frac;
    int restart_init;
    int path;              // prediction kernel: 0 = tcgen05 screen, 1 = FP32 form
};

// Source splits of target tile a of the symmetric screen: its L source tiles in ranges of
// about len (at most 8 ranges), so that the work list balances; len is the filter's
// tc_split_len (64, or shorter when the work per CTA is small).
__host__ __device__ __forceinline__ int tc_sym_splits(int L, int len) {
    const int s = (L + len - 1) / len;
    return s < 1 ? 1 : (s > 8 ? 8 : s);
}

// Launch helpers (defined in the .cu files).
template <typename T>
cudaError_t launch_sobol_dirs(const uint32_t* params, uint32_t* dirs, int r, cudaStream_t s);
cudaError_t launch_sobol_points(const uint32_t* dirs, int r, int r_pad, long long first,
                                long long count, float* u, uint32_t* bits, const double* halfwidth,
                                cudaStream_t s);
cudaError_t launch_lds_points(int kind, const uint32_t* primes, uint32_t p_faure, int r, int r_pad, long long n,
                              float* u, const double* halfwidth, cudaStream_t s);

int prep_grid(long long n_pad);
template <typename T>
cudaError_t launch_prep(const Consts<T>& k, const Bufs<T>& b, bool init_weights, bool first,
                        double prior_mean, double prior_var, cudaStream_t s);

template <typename T>
cudaError_t launch_ksum_simt(const Consts<T>& k, const Bufs<T>& b, cudaStream_t s, int* launches = nullptr);
cudaError_t launch_ksum_scr32(const Consts<float>& k, const Bufs<float>& b, int k1, cudaStream_t s);
cudaError_t launch_op_build(const Consts<float>& k, const Bufs<float>& b, bool force, cudaStream_t s);
cudaError_t launch_op_apply(const Consts<float>& k, const Bufs<float>& b, cudaStream_t s);
cudaError_t prepare_op_apply();
cudaError_t launch_ksum_tc(const Consts<float>& k, const Bufs<float>& b, cudaStream_t s,
                           int* launches);
size_t tc_scratch_bytes(long long n_pad);
cudaError_t prepare_ksum_tc();
int tc_choose_splits(long long tiles, int nst, int grid);
int tc_pair_max_clusters();
int tc_max_split();

template <typename T>
cudaError_t launch_record(const Consts<T>& k, const Bufs<T>& b, double* hist_row, cudaStream_t s);

template <typename T>
cudaError_t launch_update(const Consts<T>& k, const Bufs<T>& b, const double* dy,
                          int restart_interval, double ess_frac, cudaStream_t s, int* launches);

template <typename T>
cudaError_t launch_restart(const Consts<T>& k, const Bufs<T>& b, int mode, int init_kind, double base_R,
                           struct ::yy_mlp* net, cudaStream_t s, int* launches);

template <typename T>
cudaError_t launch_normalise_only(const Consts<T>& k, const Bufs<T>& b, cudaStream_t s,
                                  int* launches);
template <typename T>
cudaError_t launch_update_shard(const Consts<T>& k, const Bufs<T>& b, const double* dy, double* rec, cudaStream_t s,
                                int* launches);

size_t part_bytes(int r_pad);

cudaError_t launch_sobol_points_restart(const uint32_t* dirs, int r, int r_pad, long long n, float* u,
                                        const double* next_half, const DevStats* st, cudaStream_t s);
cudaError_t mlp_propose(struct ::yy_mlp* net, int r, const double* mean, const double* var, const double* dy,
                        const double* centre, double dt, const int* flag, cudaStream_t s, int* launches);
const float* mlp_output(const struct ::yy_mlp* net);

// Batched launches: one launch covers every trajectory (grid.y = trajectory).
template <typename T>
cudaError_t launch_update_batch(const Traj<T>* d_traj, int B, int r_max, const double* dy_row,
                                int nbu, cudaStream_t s, int* launches);
template <typename T>
cudaError_t launch_restart_batch(const Traj<T>* d_traj, int B, int r_max, long long n_pad_max,
                                 int nbu, cudaStream_t s, int* launches);
template <typename T>
cudaError_t launch_record_batch(const Traj<T>* d_traj, int B, double* hist_row, cudaStream_t s, int* launches);
template <typename T>
cudaError_t launch_reset_batch(const Traj<T>* d_traj, int B, cudaStream_t s, int* launches);
bool make_tc_map(void* map /* CUtensorMap */, const void* base, long long rows, int cols, int box_rows, bool fp8);
cudaError_t launch_ksum_tc_batch(const Traj<float>* d_traj, int B, int N, long long n_pad_max,
                                 const void* d_maps /* CUtensorMap[2B] */, const int4* d_items,
                                 const int* d_cta_start, int grid, int bn, const Consts<float>& k_any,
                                 const Bufs<float>& b_any, const void* map_any, cudaStream_t s, int* launches);

template <typename T>
cudaError_t launch_ksum_simt_batch(const Traj<T>* d_traj, int B, int N, long long n_pad_max, int r_max,
                                   cudaStream_t s, int* launches);

}  // namespace yy
