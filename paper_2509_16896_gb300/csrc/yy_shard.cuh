// Merge of the per-shard records of a filter whose target rows are split across devices.
//
// Shard g owns an equal chunk of the target rows.  After its likelihood update it holds,
// for its rows, ell'_i normalised by its own log-sum-exp lam_g (relative to the handle's
// offsets, which are the same on every shard), and a record
//     [lam_g, W_g, Q_g, 0, mean_g[r], M2_g[r]]
// with w_i = exp(ell'_i - lam_g) over its rows: W_g = sum w_i, Q_g = sum w_i^2, mean_g the
// w-weighted mean of the box coordinates u and M2_g the w-weighted centred second moment.
// Relative to the global log-sum-exp Lambda = log sum_g W_g e^{lam_g}, shard g's weights
// scale by s_g = e^{lam_g - Lambda}, so the global sums are
//     W = sum_g s_g W_g,  Q = sum_g s_g^2 Q_g,
// and the global mean and M2 follow from Chan's parallel rule applied to the pairs
// (s_g W_g, mean_g, s_g M2_g) in shard order.  The functions below are compiled for the host
// (so the merge can be checked without a device) and for the device (the merge kernel).
#pragma once

#include <math.h>

namespace yy {

constexpr int kShardHead = 4;   // lam, W, Q, spare; then mean[r], M2[r]

__host__ __device__ inline int shard_record_len(int r) { return kShardHead + 2 * r; }

// Lambda (relative), W, Q and the scale s_g of every shard (s[G]); shards without weight
// (W_g = 0) get s_g = 0.
__host__ __device__ inline void shard_merge_scalars(const double* rec, int G, int r, double* lam, double* W,
                                                    double* Q, double* s) {
    const int L = shard_record_len(r);
    double m = -INFINITY;
    for (int g = 0; g < G; ++g) {
        const double* p = rec + (size_t)g * L;
        if (p[1] > 0.0) m = fmax(m, p[0] + log(p[1]));
    }
    double acc = 0.0;
    if (m != -INFINITY)
        for (int g = 0; g < G; ++g) {
            const double* p = rec + (size_t)g * L;
            if (p[1] > 0.0) acc += exp(p[0] + log(p[1]) - m);
        }
    const double Lam = (m == -INFINITY) ? -INFINITY : m + log(acc);
    double w = 0.0, q = 0.0;
    for (int g = 0; g < G; ++g) {
        const double* p = rec + (size_t)g * L;
        const double sg = (p[1] > 0.0 && Lam != -INFINITY) ? exp(p[0] - Lam) : 0.0;
        s[g] = sg;
        w += sg * p[1];
        q += sg * sg * p[2];
    }
    *lam = Lam;
    *W = w;
    *Q = q;
}

// Global weighted mean and M2 of coordinate d (Chan's rule over the shards in order).
__host__ __device__ inline void shard_merge_dim(const double* rec, int G, int r, const double* s, int d,
                                                double* mean, double* M2) {
    const int L = shard_record_len(r);
    double W = 0.0, mu = 0.0, m2 = 0.0;
    for (int g = 0; g < G; ++g) {
        const double* p = rec + (size_t)g * L;
        const double Wg = s[g] * p[1];
        if (!(Wg > 0.0)) continue;
        const double mg = p[kShardHead + d], M2g = s[g] * p[kShardHead + r + d];
        if (!(W > 0.0)) {
            W = Wg; mu = mg; m2 = M2g;
            continue;
        }
        const double Wn = W + Wg;
        const double delta = mg - mu;
        mu = fma(delta, Wg / Wn, mu);
        m2 += M2g + delta * delta * (W * Wg / Wn);
        W = Wn;
    }
    *mean = mu;
    *M2 = m2;
}

}  // namespace yy
