/*
 * yy.h -- C ABI of libyy, the GB300 (sm_103a) online stage of the improved Yau--Yau
 * filter (arXiv 2509.16896).
 *
 * The paper is cited by section title.  The filtering problem ("Continuous-Time Nonlinear
 * Filtering Problem", eq. NonlinearFilter) is
 *     dX = f(X) dt + dV,   dY = h(X) dt + dW,   X in R^r, Y in R^m,
 * with unit-covariance Brownian motions.  The library carries the unnormalised
 * conditional density as log-weights on n scrambled-Sobol nodes in a box
 * [c - R, c + R]^r and advances it one observation step at a time:
 *     yy_predict   prediction by the N-scale kernel operator ("Solving Kolmogorov Equations
 *                  via Low-Discrepancy Sampling and Kernel Approximation", eq.
 *                  general_kernel) in log-sum-exp form ("Log-Domain Computation")
 *     yy_update    Ito-corrected likelihood update ("Procedure for the Improved Yau-Yau
 *                  Algorithm", online stage), log-domain normalisation ("Log-Domain
 *                  Computation"), posterior mean (the procedure's step 4), variance and
 *                  effective sample size
 *     yy_estimate  copies the estimates to the host
 *     yy_restart   local resampling-restart ("Local Resampling-Restart Mechanism")
 *
 * Conventions shared by every entry point
 *   - Memory.  Device memory is owned by the caller: it passes one device workspace of at
 *     least yy_workspace_bytes() bytes (256-byte aligned) to yy_create and keeps it alive
 *     until yy_destroy.  The library never allocates or frees device memory.  The opaque
 *     yy_filter handle (host memory) is owned by the library.
 *   - Streams.  Every call is stream-ordered on the CUDA stream given to yy_create (a
 *     cudaStream_t passed as void*, NULL = legacy default stream).  Only the calls that
 *     return host data (yy_estimate, yy_get_*, yy_restart with a non-NULL report
 *     pointer) synchronise that stream; none calls cudaDeviceSynchronize.
 *   - Errors.  Every call returns a yy_status and never aborts.  Arguments are checked
 *     before any launch (YY_ERR_ARG).  Device-side conditions (non-finite normaliser,
 *     every weight zero, a wait that timed out) set a sticky status word that
 *     yy_estimate returns.
 *   - Models.  m = r; h is componentwise.  YY_MODEL_CUBIC: f(x) = cos x, h(x) = x^3.
 *     YY_MODEL_LINEAR: f(x) = a x, h(x) = x.  YY_MODEL_PAPER_E1 (the paper's large-scale
 *     scalability test, "Large-Scale Scalability Test"): f(x) = sin(x) (A x) + sin(2x) (A1 x)
 *     elementwise with A, A1 upper bidiagonal (diagonal -0.5 / -0.3,
 *     superdiagonal 0.1 / 0.3), h(x) = (x - 100)^3.
 *   - Layout.  Node coordinates are float32 box coordinates u (x = c + u), rows of
 *     r values, row-major; host arrays passed in or out are dense [n][r].
 */
#ifndef YY_H
#define YY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define YY_EXPORT __attribute__((visibility("default")))
#else
#define YY_EXPORT
#endif

#define YY_API_VERSION 1
#define YY_MAX_SCALES 4
#define YY_MAX_DIM 1024
#define YY_SOBOL_POLY_WORDS 16
#define YY_SOBOL_SCRAMBLE_WORDS 33
#define YY_NOALLOC_MAX_DIM 1024

typedef struct yy_filter yy_filter;

typedef enum {
    YY_OK = 0,
    YY_ERR_ARG = 1,          /* invalid argument; nothing was launched */
    YY_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    YY_ERR_WORKSPACE = 3,    /* workspace missing, misaligned or too small */
    YY_ERR_NONFINITE = 4,    /* the log-normaliser or an estimate is NaN or infinite */
    YY_ERR_DEGENERATE = 5,   /* every log-weight is -inf after an update */
    YY_ERR_TIMEOUT = 6,      /* a device-side wait gave up (bounded spin) */
    YY_ERR_STATE = 7,        /* call out of order (e.g. predict before init_nodes) */
    YY_ERR_UNSUPPORTED = 8   /* configuration not supported by this build */
} yy_status;

typedef enum { YY_MODEL_CUBIC = 0, YY_MODEL_LINEAR = 1, YY_MODEL_PAPER_E1 = 2 } yy_model;

/* Node sets (Appendix A): scrambled Sobol (yy_init_nodes), or Halton / Faure
 * (yy_init_nodes_lds), the paper's choices for low dimension. */
typedef enum { YY_NODES_SOBOL = 0, YY_NODES_HALTON = 1, YY_NODES_FAURE = 2 } yy_nodes;

/* Arithmetic of the prediction step.  FP64: every step in float64.  FP32: exact
 * float32 differences over every pair.  BF16: a tcgen05 BF16 Gram product screens out pairs
 * whose kernel term is provably negligible, and the remaining pairs are evaluated exactly
 * in float32 (results agree with FP32 within float32 rounding).  FP32_SCREEN: the same kind
 * of screen on the FMA pipes, no tensor cores: a tile of 64 x 64 pairs is skipped when the
 * exact float32 squared distance of every live pair over the first 64 k coordinates
 * (k = screen_prefix, default half of the 64-coordinate chunks) exceeds the row's screening
 * radius; every other tile is evaluated exactly as in FP32 (results agree with FP32 within
 * float32 rounding).  Not accepted by batches. */
typedef enum { YY_PREC_FP64 = 0, YY_PREC_FP32 = 1, YY_PREC_BF16 = 2, YY_PREC_FP32_SCREEN = 3 } yy_precision;

/* Log-weights after a restart ("Local Resampling-Restart Mechanism" only says that the
 * filter restarts at x_hat):
 * GAUSS = log N(x; x_hat, diag(max(v_hat, (R/4)^2))), UNIFORM = equal weights. */
typedef enum { YY_RESTART_INIT_GAUSS = 0, YY_RESTART_INIT_UNIFORM = 1 } yy_restart_init;

/* Where a restart puts the new box.  PLAIN: centre x_hat, half-widths unchanged ("Local
 * Resampling-Restart Mechanism").  LEARNED: centre x_hat + delta and half-widths R exp(lambda) from the restart-proposal
 * network attached with yy_set_restart_mlp (a library addition, not in the paper); it falls
 * back to PLAIN when no network is attached, when an output is not finite, when a
 * half-width leaves [R/8, 8R], or when the box would not contain x_hat. */
typedef enum { YY_RESTART_PLAIN = 0, YY_RESTART_LEARNED = 1 } yy_restart_rule;

/* Operands of the screening Gram product of the BF16 prediction (library design, not in the
 * paper): BF16 (error bound 2^-6 |u_i||u_s|), or FP8 e4m3 with the coordinates scaled by a
 * power of two (bound 0.135 |u_i||u_s| plus a term for subnormal coordinates; twice the
 * tensor rate, half the operand bytes, first-pass chunks of 128 coordinates). */
typedef enum { YY_SCREEN_BF16 = 0, YY_SCREEN_FP8 = 1 } yy_screen_type;

/* Noise coefficients (Section "General Nonlinear Filtering with Noise Coefficients"):
 * dX = f dt + U(X) dV, dY = h dt + V(X) dW.  UNIT: U = V = I.  DIAG: diagonal and
 * state-dependent, U_d(x) = noise_u (1 + noise_u_kappa sin^2 x_d), zero for the first
 * noise_u_zero coordinates (then a = U U^T is singular and its pseudo-inverse is used),
 * V_d(x) = noise_v (1 + noise_v_kappa sin^2 x_d).  The kernel takes the metric a(x)^+ of the
 * target and -1/2 log det_+ a(x) (the table's kernel row, as printed: its prefactor keeps
 * (2 pi dt)^(-r/2)); the update weighs h and dy by b(x)^-1.  DIAG runs in FP64 and FP32
 * precision with the cubic or linear model; other combinations return YY_ERR_UNSUPPORTED
 * from yy_create. */
typedef enum { YY_NOISE_UNIT = 0, YY_NOISE_DIAG = 1 } yy_noise;

/* yy_restart modes: AUTO applies the device-side test computed by the last yy_update
 * (ESS < ess_frac * n, or restart_interval >= 2 and step % restart_interval == 0);
 * FORCE restarts unconditionally; NEVER only reports the test. */
typedef enum { YY_RESTART_AUTO = 0, YY_RESTART_FORCE = 1, YY_RESTART_NEVER = 2 } yy_restart_mode;

typedef struct {
    int32_t r;                 /* state dimension, 1..YY_MAX_DIM */
    int32_t m;                 /* observation dimension; must equal r */
    int64_t n;                 /* nodes, >= 2 */
    double dt;                 /* step, > 0 */
    double R;                  /* default box half-width, > 0 */
    int32_t n_scales;          /* N of eq. general_kernel, 1..YY_MAX_SCALES; s_j = 2^(j-1) */
    int32_t model;             /* yy_model */
    double model_a;            /* drift slope of YY_MODEL_LINEAR */
    int32_t precision;         /* yy_precision */
    int32_t restart_interval;  /* iota; <= 1: no interval restart */
    double ess_frac;           /* restart when ESS < ess_frac * n; 0 disables */
    int32_t restart_init;      /* yy_restart_init */
    double prior_mean;         /* x_0 ~ N(prior_mean, prior_var I) */
    double prior_var;          /* > 0 */
    int32_t restart_rule;      /* yy_restart_rule */
    int32_t screen_prefix;     /* YY_PREC_BF16 only: coordinates of the first screening pass
                                * of the prediction, in stages of 64 (BF16 screen) or 128 (FP8
                                * screen) coordinates (see yy_predict); 0 =
                                * chosen on the device from the previous predictions
                                * (default), k >= 1 = fixed (values >= ceil(r/64) give one
                                * full-coordinate pass), < 0 invalid. Members of a batch
                                * default to one full-coordinate pass. Results do not depend
                                * on it beyond float32 rounding. */
    int32_t screen_type;       /* YY_PREC_BF16 only: yy_screen_type, the operand type of the
                                * screen's Gram product. Results do not depend on it beyond
                                * float32 rounding (the screen's bound covers the operand
                                * rounding). */
    int32_t noise;             /* yy_noise (0 = unit noise) */
    int32_t noise_u_zero;      /* DIAG: leading coordinates without state noise, 0..r */
    double noise_u, noise_u_kappa;   /* DIAG: U_d(x) = noise_u (1 + noise_u_kappa sin^2 x_d); > 0, >= 0 */
    double noise_v, noise_v_kappa;   /* DIAG: V_d(x) = noise_v (1 + noise_v_kappa sin^2 x_d); > 0, >= 0 */
    int32_t materialise;       /* float precisions, single filters: 0 = the prediction recomputes its
                                * kernel sums every step; 1 = the workspace also holds the
                                * materialised per-scale log-operator (N n_pad^2 floats) and
                                * yy_tune_materialise chooses between the two schedules (recompute
                                * until it is called); 2 = always the materialised operator */
} yy_config;

/* Bytes of device workspace that yy_create needs for cfg (0 if cfg is invalid). */
YY_EXPORT size_t yy_workspace_bytes(const yy_config* cfg);

/* Creates a filter on the current CUDA device.  d_workspace: device pointer,
 * 256-byte aligned, >= yy_workspace_bytes(cfg) bytes, owned by the caller.
 * stream: cudaStream_t or NULL.  *out receives the handle. */
YY_EXPORT yy_status yy_create(const yy_config* cfg, void* d_workspace, size_t bytes, void* stream,
                    yy_filter** out);

/* Releases the host handle (the workspace stays the caller's). NULL is accepted. */
YY_EXPORT yy_status yy_destroy(yy_filter* f);

/* Node generation ("Sobol Sequence" in the appendix "Low-Discrepancy Sequence Sampling";
 * step 1 of "Procedure for the Improved Yau-Yau Algorithm"): generates the n scrambled
 * Sobol points on the device and maps them to the box, then evaluates the prior
 * log-weights log sigma_0 and the Dirichlet mask ("Algorithm for Kolmogorov Equation",
 * steps 4 and 3).
 *   h_poly      host uint32 [r][YY_SOBOL_POLY_WORDS]: per dimension the degree s of its
 *               primitive polynomial (0 = identity dimension), the inner coefficients a
 *               (a_1 most significant), then m_1..m_s.
 *   h_scramble  host uint32 [r][YY_SOBOL_SCRAMBLE_WORDS] or NULL (no scramble): rows
 *               1..32 of a lower-triangular unit-diagonal GF(2) matrix (row k acts on
 *               output digit k, stored at bit 32-k), then the digital shift.
 *   h_center    host double [r], box centre c.
 *   h_halfwidth host double [r] or NULL (all equal to cfg.R).
 * Coordinates: u = R_d (2 (y + 1/2) 2^-32 - 1) in float64, rounded to float32, where y is
 * the scrambled 32-bit integer of point i (indices 0..n-1, Gray-code order). */
YY_EXPORT yy_status yy_init_nodes(yy_filter* f, const uint32_t* h_poly, const uint32_t* h_scramble,
                        const double* h_center, const double* h_halfwidth);

/* Node generation with Halton or Faure points (Appendix A, "Halton Sequence", "Faure
 * Sequence"), otherwise as yy_init_nodes (prior weights, Dirichlet mask).  kind:
 * YY_NODES_HALTON (coordinate d: radical inverse in the d-th prime) or YY_NODES_FAURE (one
 * base, the smallest prime >= r; generator matrices the powers of the Pascal matrix mod
 * that base).  Point i of the node set is sequence index i + 1 (index 0 is the corner of
 * the box).  Coordinates u = R_d (2 phi - 1) in float64, rounded to float32, phi the point's
 * coordinate in [0, 1) evaluated exactly (digit integer over p^M, p^M <= 2^53, one rounding).
 * h_center, h_halfwidth as for yy_init_nodes.  A filter with these nodes does not take the
 * learned restart (its re-mapping of nodes is defined for Sobol points): yy_set_restart_mlp
 * then returns YY_ERR_UNSUPPORTED. */
YY_EXPORT yy_status yy_init_nodes_lds(yy_filter* f, int32_t kind, const double* h_center, const double* h_halfwidth);

/* Writes the scrambled Sobol integers of points first..first+count-1 to d_bits
 * (device uint32 [count][r], caller-owned).  Same generator as yy_init_nodes. */
YY_EXPORT yy_status yy_sobol_bits(yy_filter* f, uint32_t* d_bits, int64_t first, int64_t count);

/* Prediction ("Solving Kolmogorov Equations via Low-Discrepancy Sampling and Kernel
 * Approximation", eq. general_kernel; the prediction step of "Log-Domain Computation"):
 *   ell_pred(i) = log( sum_j c_j e^{L_j(i)} + c_{N+1} e^{ell(i)} ),
 *   L_j(i) = log sum_{s unmasked} K_{dt/s_j}(x_i, x_s) w_q e^{ell(s)},
 * K the first-order kernel of eq. kernel, w_q = prod_d 2 R_d / n, c the solution of the
 * generalised Vandermonde system.  Boundary nodes get -inf.  A non-positive combination
 * gives -inf and is counted.  Asynchronous.
 * YY_PREC_BF16: pairs are screened on the tensor cores by a lower bound of |u_i - u_s|
 * (a BF16 Gram product with a rigorous error bound) and only pairs that can carry more
 * than e^-20 of a row's sum are evaluated exactly in float32.  The first screening pass
 * uses the first 64 k coordinates (k = cfg.screen_prefix, or chosen on the device);
 * |u_i - u_s| restricted to them is still a lower bound.  Tiles in which that pass leaves
 * many candidates are screened again with all coordinates. */
YY_EXPORT yy_status yy_predict(yy_filter* f);

/* Correction and estimate ("Procedure for the Improved Yau-Yau Algorithm", online stage
 * and step 4; "Log-Domain Computation"):
 *   ell'(i) = ell_pred(i) + h(x_i).dy - dt/2 |h(x_i)|^2,  Lambda = LSE ell',
 *   normalised weights, x_hat = sum w x, v_hat = sum w (x - x_hat)^2, ESS = 1/sum w^2,
 *   Z += Lambda, then the restart test.
 * d_dy: device double [m], the observation increment y(tau_k) - y(tau_{k-1}).
 * Asynchronous. */
YY_EXPORT yy_status yy_update(yy_filter* f, const double* d_dy);

/* Copies the last step's estimate to the host (any pointer may be NULL):
 * h_mean, h_var double [r]; h_ess, h_lognorm (Z_k) double.  Synchronises the stream
 * and returns the sticky device status. */
YY_EXPORT yy_status yy_estimate(yy_filter* f, double* h_mean, double* h_var, double* h_ess,
                      double* h_lognorm);

/* Local resampling-restart ("Local Resampling-Restart Mechanism"): re-centres the box at
 * x_hat, keeps the reference node set (translation), re-evaluates the drift at the new nodes and re-initialises the
 * log-weights (cfg.restart_init).  mode: yy_restart_mode.  h_did_restart: NULL (stay
 * asynchronous) or a host int32 that receives 1 if a restart happened (synchronises). */
YY_EXPORT yy_status yy_restart(yy_filter* f, int32_t mode, int32_t* h_did_restart);

/* Runs K filter steps back to back on the handle's stream, without host round trips:
 * for each k, yy_predict, yy_update with d_dy_all + k m, an optional record of the
 * estimate, and yy_restart(YY_RESTART_AUTO).
 *   d_dy_all  device double [K][m], observation increments of the K steps
 *   d_hist    device double [K][2r + 4] or NULL; row k receives x_hat[r], v_hat[r], ESS,
 *             Lambda_k, Z_k and 1.0 if the restart test fired at step k (else 0.0)
 * Asynchronous. */
YY_EXPORT yy_status yy_run_steps(yy_filter* f, const double* d_dy_all, int64_t K, double* d_hist);

/* Captures yy_run_steps(f, d_dy_all, K, d_hist) into a CUDA graph owned by the handle
 * (replacing any earlier one); nothing is executed.  The handle's stream must be a
 * created stream (not NULL / the legacy default stream).  The pointers are baked into the
 * graph: their contents may change between replays, the buffers must stay alive. */
YY_EXPORT yy_status yy_graph_capture(yy_filter* f, const double* d_dy_all, int64_t K, double* d_hist);

/* Replays the captured K-step graph on the handle's stream (asynchronous).  Returns
 * YY_ERR_STATE if nothing was captured. */
YY_EXPORT yy_status yy_graph_launch(yy_filter* f);

/* Number of kernel launches one replay of the captured graph performs (0 if none). */
YY_EXPORT int64_t yy_graph_kernel_count(const yy_filter* f);

/* ---- restart-proposal network (a library addition; the paper has no counterpart) -----
 * A perceptron z = [x_hat - c; sqrt(v_hat); dy/sqrt(dt)] (3r, c the centre of the box the
 * estimate was computed in; normalised, see
 * yy_mlp_set_input_norm) -> H -> H (ReLU) -> [delta; lambda]
 * (2r), trained and run on the device with BF16 operands and FP32 accumulation.  Loss:
 * mean over rows and coordinates of (t - delta)^2 / (2 s^2) + log s, s = (R/3) exp(lambda),
 * where t = x_true - x_hat at restarts of a plain run.  Parameters are packed FP32:
 * W1 [H][3r], b1 [H], W2 [H][H], b2 [H], W3 [2r][H], b3 [2r].  Memory: one caller-owned device
 * workspace of yy_mlp_workspace_bytes bytes (256-byte aligned). */
typedef struct yy_mlp yy_mlp;

YY_EXPORT int64_t yy_mlp_param_count(int32_t r, int32_t hidden);
YY_EXPORT size_t yy_mlp_workspace_bytes(int32_t r, int32_t hidden, int32_t max_batch);
YY_EXPORT yy_status yy_mlp_create(int32_t r, int32_t hidden, int32_t max_batch, void* d_workspace, size_t bytes,
                                  void* stream, yy_mlp** out);
YY_EXPORT yy_status yy_mlp_destroy(yy_mlp* net);

/* Copies parameters in (and resets the Adam moments) / out; host float [param_count]. */
YY_EXPORT yy_status yy_mlp_set_params(yy_mlp* net, const float* h_params);
YY_EXPORT yy_status yy_mlp_get_params(yy_mlp* net, float* h_params);

/* Input normalisation zn = clamp((z - mean) / std, -4, 4) applied before the first layer
 * (host float [3r] each, std > 0); identity (mean 0, std 1) after yy_mlp_create. */
YY_EXPORT yy_status yy_mlp_set_input_norm(yy_mlp* net, const float* h_mean, const float* h_std);

/* Forward pass: d_x device float [B][3r] -> d_out device float [B][2r]. */
YY_EXPORT yy_status yy_mlp_forward(yy_mlp* net, const float* d_x, int32_t B, float* d_out);

/* Loss and parameter gradients of one batch (B <= max_batch): d_x [B][3r], d_t [B][r];
 * R the base half-width.  h_loss (host float) and h_grads (host float [param_count]) may be
 * NULL.  Synchronises. */
YY_EXPORT yy_status yy_mlp_loss_grad(yy_mlp* net, const float* d_x, const float* d_t, int32_t B, double R,
                                     float* h_loss, float* h_grads);

/* Adam training (b1 0.9, b2 0.999, eps 1e-8) on M rows, epochs passes of shuffled
 * mini-batches (seeded); h_last_loss receives the last mini-batch's loss.  Synchronises. */
YY_EXPORT yy_status yy_mlp_train(yy_mlp* net, const float* d_x, const float* d_t, int64_t M, double R,
                                 int32_t epochs, int32_t batch, float lr, uint64_t seed, float* h_last_loss);

/* Attaches (or with NULL detaches) the network used by restarts of a filter whose
 * cfg.restart_rule is YY_RESTART_LEARNED.  The network must have been created with the
 * filter's r; it must stay alive while attached. */
YY_EXPORT yy_status yy_set_restart_mlp(yy_filter* f, yy_mlp* net);

/* ---- batches of independent filters ------------------------------------------------
 * B filters with their own r, n, model, box and restart settings (same precision, FP32 or
 * BF16, and same n_scales) advance together: every pass of a step is one launch for the
 * whole batch, the BF16 prediction is one persistent tcgen05 launch over a work list of
 * (filter, 128-target tile) items balanced longest-first across the SMs, and the K-step
 * loop can be captured as one CUDA graph.  Memory: one caller-owned device workspace of
 * yy_batch_workspace_bytes(cfgs, B) bytes (256-byte aligned) holds the descriptors and
 * every filter's workspace. */
typedef struct yy_batch yy_batch;

YY_EXPORT size_t yy_batch_workspace_bytes(const yy_config* cfgs, int32_t B);

/* Creates the batch and its B filter handles (owned by the batch). */
YY_EXPORT yy_status yy_batch_create(const yy_config* cfgs, int32_t B, void* d_workspace, size_t bytes,
                                    void* stream, yy_batch** out);
YY_EXPORT yy_status yy_batch_destroy(yy_batch* bt);

/* Borrows filter b (0 <= b < B) for yy_init_nodes, yy_estimate, yy_get_* and yy_set_state.
 * Every filter must have had yy_init_nodes before the first batched step. */
YY_EXPORT yy_status yy_batch_filter(yy_batch* bt, int32_t b, yy_filter** out);

/* K batched steps (prediction, correction, estimate, automatic restart of every filter).
 *   d_dy_all  device double [K][M], M = sum_b m_b; filter b's increments at offset
 *             sum_{b' < b} m_b' of each row
 *   d_hist    device double [K][H] or NULL, H = sum_b (2 r_b + 4); filter b's record
 *             (x_hat, v_hat, ESS, Lambda, Z, restart flag) at offset sum_{b' < b} (2 r_b' + 4)
 * Asynchronous (the first call uploads the descriptors and synchronises once). */
YY_EXPORT yy_status yy_batch_run_steps(yy_batch* bt, const double* d_dy_all, int64_t K, double* d_hist);

/* One batched prediction (all filters), for timing; leaves every filter "predicted". */
YY_EXPORT yy_status yy_batch_predict(yy_batch* bt);

/* Captures yy_batch_run_steps(bt, d_dy_all, K, d_hist) as a CUDA graph (needs a created
 * stream); yy_batch_graph_launch replays it. */
YY_EXPORT yy_status yy_batch_graph_capture(yy_batch* bt, const double* d_dy_all, int64_t K, double* d_hist);
YY_EXPORT yy_status yy_batch_graph_launch(yy_batch* bt);

/* Schedule of the batched BF16 prediction: source-tile width bn (128 or 256) and the
 * number of persistent CTAs (1..1024).  yy_batch_autotune first runs one prediction with
 * every filter on the tensor-core screen and reads each filter's screen pass fraction
 * (pairs evaluated exactly / n^2); it then times, on the batch itself (reps predictions
 * each), the routing thresholds {3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1, never} (filters whose
 * fraction exceeds it use the FP32 form, which is faster when most pairs are within reach
 * of the kernel, i.e. at low r) with bn = 256 and grid = 2 x SM count, then bn in
 * {256, 128} x grid in {1, 2, 4} x SM count with the best routing, and keeps the fastest.
 * If cache_path is not NULL the choice is recorded there keyed by
 * the batch's shape and reused instead of timing.  yy_batch_get_routing reports the
 * per-filter choice (0 = tensor-core screen, 1 = FP32 form; host int32 [B]). */
YY_EXPORT yy_status yy_batch_set_schedule(yy_batch* bt, int32_t bn, int32_t grid);
YY_EXPORT yy_status yy_batch_get_schedule(const yy_batch* bt, int32_t* h_bn, int32_t* h_grid);
YY_EXPORT yy_status yy_batch_autotune(yy_batch* bt, const char* cache_path, int32_t reps, int32_t* h_bn,
                                      int32_t* h_grid);
YY_EXPORT yy_status yy_batch_get_routing(const yy_batch* bt, int32_t* h_path);
/* Fixes the per-filter prediction path (host int32 [B]: 0 = tensor-core screen, allowed only
 * for BF16 precision; 1 = FP32 form), replacing the autotuner's routing.  Results agree
 * within float32 rounding either way. */
YY_EXPORT yy_status yy_batch_set_routing(yy_batch* bt, const int32_t* h_path);

/* Kernel launches issued so far, and per replay of the captured graph. */
YY_EXPORT int64_t yy_batch_launch_count(const yy_batch* bt);
YY_EXPORT int64_t yy_batch_graph_kernel_count(const yy_batch* bt);

/* Copies node coordinates u (host float [n][r]) and/or the Dirichlet mask (host uint8
 * [n]); either pointer may be NULL.  Synchronises. */
YY_EXPORT yy_status yy_get_nodes(yy_filter* f, float* h_u, uint8_t* h_mask);

/* Copies the current log-weights: after yy_update (or init/restart) the normalised
 * ell_hat; after yy_predict the predicted ell_pred minus *h_offset.  h_logw is host float
 * [n] (FP32/BF16 precision) or double [n] (FP64 precision).  Synchronises. */
YY_EXPORT yy_status yy_get_log_weights(yy_filter* f, void* h_logw, double* h_offset);

/* Overwrites the filter state: box centre (host double [r]), normalised log-weights
 * (host float or double [n], as for yy_get_log_weights), running log-normaliser Z and
 * step counter.  Re-evaluates the drift at the nodes.  Used for checkpoint/resume. */
YY_EXPORT yy_status yy_set_state(yy_filter* f, const double* h_center, const void* h_logw,
                       double lognorm, int64_t step);

/* Reads the current box: centre and half-widths (host double [r] each, either may be
 * NULL).  Synchronises. */
YY_EXPORT yy_status yy_get_box(yy_filter* f, double* h_center, double* h_halfwidth);

/* Reads the box centre (host double [r]), Z and step counter. Synchronises. */
YY_EXPORT yy_status yy_get_state(yy_filter* f, double* h_center, double* h_lognorm, int64_t* h_step);

/* Number of targets whose multi-scale combination was non-positive (set to -inf) in the
 * last yy_predict.  Synchronises. */
YY_EXPORT yy_status yy_get_clamps(yy_filter* f, int64_t* h_clamps);

/* Weighted moments of node rows without any device allocation.  The paper has no
 * counterpart: this is a library service for callers that cannot allocate device memory
 * when they need the result (inside host callbacks or stream work where cudaMalloc is not
 * allowed, plug-ins whose host owns every device buffer and passes only inputs and
 * outputs, real-time loops that forbid allocation after start-up).  It computes what
 * yy_update's normalisation and estimate compute, for caller-supplied rows:
 *   w_i = exp(logw_i - LSE(logw)),  mean_d = sum_i w_i u_id,
 *   var_d = sum_i w_i (u_id - mean_d)^2,  ESS = (sum w)^2 / sum w^2.
 *   d_u     device float [n][ld], rows of r coordinates (ld >= r)
 *   d_logw  device float [n], log-weights with any common offset (-inf allowed)
 *   d_out   device double [2r + 3]: mean[r], var[r], ESS, LSE(logw), sum of weights
 *   stream  cudaStream_t or NULL
 * If every log-weight is -inf the output reads LSE = -inf with weight sum, ESS, mean and
 * variance 0 (the call is asynchronous, so this is reported in the output, not as a code).
 * Limits: 1 <= r <= YY_NOALLOC_MAX_DIM and n >= 1; anything else returns YY_ERR_ARG
 * before any launch.  YY_ERR_CUDA reports a failure of this call's own launches only.
 * Scratch lives in a fixed device array of about 2 MB inside the
 * library, held by every GPU that loads it until the process exits.  The first call on a
 * device looks up that array's device address; make it before any stream capture.  All
 * calls share the array: calls that overlap on the GPU race and must be serialised by
 * the caller.  Asynchronous; no device memory is allocated or freed. */
YY_EXPORT yy_status yy_weighted_moments_static(const float* d_u, int64_t n, int32_t r, int64_t ld,
                                               const float* d_logw, double* d_out, void* stream);

/* Limit of every bounded device-side wait in this handle's prediction kernel (the
 * tensor-core screen's pipeline waits), in seconds, 0 < seconds <= 3600; default 4 s.  When
 * a wait runs out the kernel stops, records YY_ERR_TIMEOUT in the sticky status word (read
 * by yy_estimate), lets its own copies and tensor-core work finish and returns; the
 * predicted weights of that call are not valid and the handle should be recreated.  Takes
 * effect for launches issued (or graphs captured) after the call.  A library service with
 * no counterpart in the paper: it lets a caller bound how long a stalled launch can hold
 * the GPU, and lets a test make a wait expire. */
YY_EXPORT yy_status yy_set_wait_limit(yy_filter* f, double seconds);

/* Whether the tensor-core prediction (YY_PREC_BF16) may run on pairs of CTAs (on = 1) or
 * on single CTAs (on = 0, the default).  A pair is a 2-CTA cluster on two SMs: each CTA
 * holds 128 target rows and stages half of every 256-wide source tile, and one
 * tcgen05.mma.cta_group::2 per K step computes both CTAs' Gram blocks, so each source tile
 * is fetched into shared memory once per 256 targets instead of once per 128 (a library
 * design, not in the paper).  Pairs are used when allowed and when the device can place
 * the clusters; both forms take the same screening decisions and give the same predicted
 * weights up to float32 rounding.  h_pairs (host int32, may be NULL) receives the number
 * of CTA pairs (clusters) of the handle's current schedule, 0 when it uses single CTAs.
 * Rebuilds the work list (synchronous) if nodes exist; call it outside stream capture.
 * YY_ERR_ARG for on not in {0, 1}. */
YY_EXPORT yy_status yy_set_cta_pair(yy_filter* f, int32_t on, int32_t* h_pairs);

/* The materialised schedule of the prediction (the paper's offline operator and online
 * matrix-vector product, Sections "Algorithm for Kolmogorov Equation" and "CPU/GPU
 * Parallel Acceleration", in its log-domain form, Section "Log-Domain Computation"):
 * per scale j the matrix A_j(i, s) = -|u_i - tau_j f_i - u_s|^2 / (2 tau_j) (the pair part of
 * log K_{tau_j}, float32, [N][n_pad][n_pad]) is built once per node set -- on the device at
 * the first prediction after a restart or a state change, so graphs replay it correctly --
 * and each prediction is the log-sum-exp product L_j(i) = C_j - tau_j div f_i +
 * LSE_s(A_j(i, s) + ell_s), combined across scales as in yy_predict.  The paper applies
 * one combined operator; with the negative coefficients of the multi-scale kernel its
 * logarithm is not defined everywhere, so the scales are kept apart (results equal the
 * recomputed ones within float32 rounding).
 * yy_tune_materialise times, on the handle's current state (reps launches each), the
 * recomputed prediction, the build and the apply, and chooses the materialised schedule
 * when build + m apply < m recompute, m = predicts_per_build (the predictions a node set
 * serves between restarts: the restart interval when restarts are by interval only).
 * h_ms (host double [3], may be NULL) receives the three times in ms, *h_choice 1 when the
 * materialised schedule was chosen.  Needs cfg.materialise >= 1.  Synchronous. */
YY_EXPORT yy_status yy_tune_materialise(yy_filter* f, int32_t predicts_per_build, int32_t reps, double* h_ms,
                                        int32_t* h_choice);

/* Routing of a BF16 filter's prediction (no counterpart in the paper; the paper evaluates
 * every pair): the screened tensor-core form of yy_predict, or the plain float32 form of
 * YY_PREC_FP32 (every pair, same results within float32 rounding).  The screen wins where
 * it proves most pairs negligible; where the weights spread over many nats (the paper's
 * large-scale workload) nearly every pair survives it and the plain form is faster.
 * yy_set_route: plain = 1 routes to the plain form, 0 back to the screen (the default).
 * The plain form reads the drift f of every node, which the preparation pass then stores
 * (recomputed here for the current nodes when it was not stored).
 * yy_tune_route times, on the handle's current state, reps predictions of each form (after
 * one untimed prediction of each) and keeps the faster; h_ms (host double [2], may be NULL)
 * receives the screened and plain times in ms, *h_route (may be NULL) 1 when the plain form
 * was chosen.  The timing predictions leave the weights as they were; they do advance the
 * adaptive first-pass controller of the screen.  Synchronous.  A captured graph keeps the
 * route it was captured with.
 * Both: YY_ERR_UNSUPPORTED unless the precision is YY_PREC_BF16, YY_ERR_STATE between a
 * prediction and its update, YY_ERR_ARG for plain not in {0, 1} or reps < 1. */
YY_EXPORT yy_status yy_set_route(yy_filter* f, int32_t plain);
YY_EXPORT yy_status yy_tune_route(yy_filter* f, int32_t reps, double* h_ms, int32_t* h_route);

/* Kernel launches issued by this handle so far (for launch accounting). */
YY_EXPORT int64_t yy_launch_count(const yy_filter* f);

/* Work counters of the last yy_predict: non-positive combinations (as yy_get_clamps) and,
 * for BF16 precision, the pairs that passed the screen and were evaluated exactly in
 * float32 (self terms not included).  Synchronises. */
YY_EXPORT yy_status yy_get_counters(yy_filter* f, int64_t* h_clamps, int64_t* h_exact_pairs);

/* Screen of the last BF16 yy_predict (no counterpart in the paper; work accounting of the
 * screening passes described at yy_predict): *h_last_prefix = coordinate stages of its
 * first pass (64 coordinates per stage with BF16 operands, 128 with FP8; 0 before the
 * first prediction), *h_next_prefix = those the next
 * prediction will use, *h_tiles = 128-target x source-tile blocks screened (256 sources per
 * tile for a single filter), *h_rescreened = blocks screened again over all coordinates.
 * Any pointer may be NULL.  YY_ERR_UNSUPPORTED for other precisions.  Synchronises. */
YY_EXPORT yy_status yy_get_screen(yy_filter* f, int32_t* h_last_prefix, int32_t* h_next_prefix,
                                  int64_t* h_tiles, int64_t* h_rescreened);

/* ---- one filter across several devices (target rows split, source set replicated) -----
 * Every device holds a handle of the same configuration with the same nodes; each owns an
 * equal chunk of the target rows.  Per step and device: yy_predict (the shard's rows against
 * all sources), yy_update_shard, an all-gather of every shard's rows and of every shard's
 * record by the caller (e.g. NCCL), yy_merge_shards, then yy_estimate / yy_restart as for a
 * whole filter (every device takes the same restart from the same merged estimate).  The
 * split is a library design for the prediction's n x n work; the paper has no multi-device
 * form.  yy_run_steps and CUDA-graph capture are refused while a handle is a shard of more
 * than one. */

/* Makes the handle shard `rank` of `count` (1..64): target rows
 * [rank n_pad / count, (rank + 1) n_pad / count) intersected with [0, n), n_pad = n rounded
 * up to 256; n_pad must be a multiple of 256 count.  count = 1 restores the whole filter.
 * Call between steps (not after yy_predict or yy_update_shard).  Synchronous (rebuilds the
 * tensor-core work list for the shard's tiles; a shard screens its tiles against every
 * source tile, without the symmetric blocks of a whole filter). */
YY_EXPORT yy_status yy_set_shard(yy_filter* f, int32_t rank, int32_t count);

/* First row of the handle's chunk and the chunk length n_pad / count (rows); host int64. */
YY_EXPORT yy_status yy_shard_rows(const yy_filter* f, int64_t* h_row0, int64_t* h_chunk);

/* Likelihood update of the shard's rows ("Procedure for the Improved Yau-Yau Algorithm",
 * online stage; "Log-Domain Computation").  Writes
 *   d_rows_out    device float [chunk] (double for FP64 precision): the chunk's log-weights
 *                 ell'_i - lam_g, normalised by the shard's own log-sum-exp lam_g (-inf for
 *                 padding rows)
 *   d_record_out  device double [2r + 4]: lam_g, W_g, Q_g, 0, mean_g[r], M2_g[r], with
 *                 w_i = exp(ell'_i - lam_g) over the shard's rows: W_g = sum w_i,
 *                 Q_g = sum w_i^2, mean_g and M2_g the w-weighted mean and centred second
 *                 moment of the box coordinates u
 * d_dy as for yy_update.  Asynchronous. */
YY_EXPORT yy_status yy_update_shard(yy_filter* f, const double* d_dy, void* d_rows_out, double* d_record_out);

/* Completes the step from the gathered buffers: d_rows_all device [n_pad] (shard g's chunk at
 * offset g chunk), d_records device double [count][2r + 4] in shard order.  Merges the records
 * (Lambda = log sum_g W_g e^{lam_g}, each shard's sums rescaled by e^{lam_g - Lambda}, means
 * and second moments combined by Chan's rule in shard order), sets Lambda_k, Z_k, x_hat,
 * v_hat, ESS and the restart test as yy_update does, and stores every row's normalised
 * log-weight.  count must equal the handle's shard count.  Asynchronous. */
YY_EXPORT yy_status yy_merge_shards(yy_filter* f, const void* d_rows_all, const double* d_records, int32_t count);

/* The same merge on the host (no device): h_records double [count][2r + 4] ->
 * h_out double [2r + 4] = Lambda (relative to the shards' common offset), W, Q, ESS = W^2/Q,
 * mean of u [r], variance [r]. */
YY_EXPORT yy_status yy_merge_records_host(const double* h_records, int32_t count, int32_t r, double* h_out);

/* Human-readable name of a status code (static storage). */
YY_EXPORT const char* yy_status_str(yy_status s);

#ifdef __cplusplus
}
#endif
#endif /* YY_H */
