/*
 * FP64 oracle core: the prediction step's kernel sums, written out directly.
 *
 * ORACLE / TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code with the CUDA path.
 *
 * For every target node x_i and bandwidth tau (one per scale of the multi-scale
 * kernel), this computes
 *
 *     L_tau(i) = log( sum_{s unmasked} K_tau(x_i, x_s) * w_q * exp(ell_s) )
 *
 * with the first-order kernel (eq. kernel, "First-Order Kernel Construction"),
 *
 *     log K_tau(x, y) = -(r/2) log(2 pi tau) - |x - y|^2 / (2 tau)
 *                       - (y - x) . f(x) - (tau/2) (2 div f(x) + |f(x)|^2),
 *
 * where x (first argument) is the evaluation point and y the integration variable
 * (Remark after eq. L_Delta_t); with state-dependent noise coefficients (Section "General
 * Nonlinear Filtering with Noise Coefficients", kernel row of its table) the squared norms
 * and the inner product take the metric a(x)^-1 (its pseudo-inverse when a(x) is singular)
 * of the evaluation point and log K gains -1/2 log det a(x) (det over the positive
 * eigenvalues); here a(x) is diagonal, passed as minv[i][d] = 1/a_d(x_i) (0 where
 * a_d(x_i) = 0) and hld[i] = 1/2 sum log a_d(x_i) over the positive a_d.  And w_q = prod_d (2 R_d) / n is the quadrature
 * volume per node that turns the integral into a sum over the nodes (the "Delta y"
 * factor of that Remark).  The sum is a log-sum-exp ("Log-Domain Computation", Prediction Step),
 * taken by the two-pass definition max + log sum exp(a - max).  Differences x - y are
 * formed directly; nothing is expanded into Gram products.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/*
 * n, r        : node count and state dimension
 * x           : [n][r] node positions (row-major)
 * fx          : [n][r] drift f(x_i)
 * divf        : [n]    divergence of f at x_i
 * logw        : [n]    log-weights ell_s of the sources
 * mask        : [n]    1 = node on the Dirichlet boundary (excluded as a source)
 * n_tau, tau  : bandwidths
 * log_wq      : log of the quadrature volume per node
 * t0, t1      : targets t0 <= i < t1 are evaluated
 * out         : [(t1 - t0)][n_tau] results L_tau(i); -inf when no source contributes
 * n_threads   : OpenMP threads (<= 0: library default)
 * minv, hld   : [n][r] and [n] metric of diagonal noise coefficients, or NULL (unit noise)
 */
void yyo_kernel_lse(int64_t n, int32_t r, const double* x, const double* fx,
                    const double* divf, const double* logw, const uint8_t* mask,
                    int32_t n_tau, const double* tau, double log_wq,
                    int64_t t0, int64_t t1, double* out, int32_t n_threads,
                    const double* minv, const double* hld)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const double log_2pi = log(2.0 * M_PI);
#pragma omp parallel
    {
        double* terms = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = t0; i < t1; ++i) {
            const double* xi = x + (size_t)i * r;
            const double* fi = fx + (size_t)i * r;
            const double* mi = minv ? minv + (size_t)i * r : NULL;
            double ff = 0.0;
            for (int32_t d = 0; d < r; ++d) ff += (mi ? mi[d] : 1.0) * fi[d] * fi[d];
            for (int32_t q = 0; q < n_tau; ++q) {
                const double t = tau[q];
                const double log_c = -0.5 * r * (log_2pi + log(t)) - (hld ? hld[i] : 0.0);
                const double tail = 0.5 * t * (2.0 * divf[i] + ff);
                double mx = -INFINITY;
                for (int64_t s = 0; s < n; ++s) {
                    if (mask[s] || isinf(logw[s])) { terms[s] = -INFINITY; continue; }
                    const double* xs = x + (size_t)s * r;
                    double d2 = 0.0, drift = 0.0;
                    for (int32_t d = 0; d < r; ++d) {
                        const double diff = xi[d] - xs[d];
                        const double m = mi ? mi[d] : 1.0;
                        d2 += m * diff * diff;
                        drift += (xs[d] - xi[d]) * m * fi[d];
                    }
                    const double logk = log_c - d2 / (2.0 * t) - drift - tail;
                    terms[s] = logk + logw[s];
                    if (terms[s] > mx) mx = terms[s];
                }
                double acc = 0.0;
                if (!isinf(mx))
                    for (int64_t s = 0; s < n; ++s) acc += exp(terms[s] - mx);
                out[(size_t)(i - t0) * n_tau + q] =
                    isinf(mx) ? -INFINITY : mx + log(acc) + log_wq;
            }
        }
        free(terms);
    }
}
