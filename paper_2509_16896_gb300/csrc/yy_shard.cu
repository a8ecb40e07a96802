// One filter with its target rows split across devices (one handle per device, each
// holding every node and its weight -- the source set is replicated -- and predicting and
// updating an equal chunk of the target rows).  Per step, on every device:
//     yy_predict          the shard's target rows against all sources
//     yy_update_shard     the shard's rows' likelihood update; its log-weights (normalised by
//                         its own log-sum-exp) and its record (yy_shard.cuh) go to caller buffers
//     all-gather          of the rows and of the records (the caller's collective)
//     yy_merge_shards     the records merged in shard order (Chan's rule with the rescaling of
//                         each shard's weights), the step's scalars and estimate set, every
//                         row's log-weight normalised by the global log-sum-exp
//     yy_restart          taken redundantly: every device has the same merged estimate
// The merge reads nothing but the gathered buffers, so every device computes the same
// result.  yy_merge_records_host runs the same merge on the host (no device needed).
#include "yy_handle.cuh"
#include "yy_shard.cuh"

namespace yy {

namespace {

constexpr int kMaxShards = 64;

// The step's scalars from the gathered records; the shard scales s_g go to b.part[0..G).
template <typename T>
__global__ void k_merge_scalars(Consts<T> k, Bufs<T> b, const double* __restrict__ rec, int G, int restart_interval,
                                double ess_frac) {
    if (threadIdx.x != 0) return;
    DevStats* st = b.stats;
    double lam, W, Q;
    shard_merge_scalars(rec, G, k.r, &lam, &W, &Q, b.part);
    if (lam == -INFINITY) {
        st->status |= kStatusDegenerate;
        lam = 0.0;
    }
    st->lam_rel = lam;
    st->wsum = W;
    st->wsq = Q;
    st->ess = (Q > 0.0) ? W * W / Q : 0.0;
    const double lam_abs = st->c_ref + st->lam_c + lam;
    st->lam = lam_abs;
    st->lognorm += lam_abs;
    if (!isfinite(lam_abs)) st->status |= kStatusNonFinite;
    st->step += 1;
    const bool by_ess = ess_frac > 0.0 && st->ess < ess_frac * (double)k.n;
    const bool by_int = restart_interval >= 2 && (st->step % restart_interval) == 0;
    st->restart_flag = (by_ess || by_int) ? 1 : 0;
}

template <typename T>
__global__ void k_merge_dims(Consts<T> k, Bufs<T> b, const double* __restrict__ rec, int G) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= k.r) return;
    double mu, m2;
    shard_merge_dim(rec, G, k.r, b.part, d, &mu, &m2);
    const double W = b.stats->wsum;
    b.mean[d] = b.centre[d] + mu;
    b.var[d] = (W > 0.0) ? m2 / W : 0.0;
    if (!isfinite(b.mean[d]) || !isfinite(b.var[d])) atomicOr(&b.stats->status, kStatusNonFinite);
}

// Row i of shard g = i / chunk holds ell'_i - lam_g; normalised: ell'_i - Lambda.
template <typename T>
__global__ void k_merge_rows(Consts<T> k, Bufs<T> b, const T* __restrict__ rows_all, const double* __restrict__ rec,
                             long long chunk) {
    const double lam = b.stats->lam_rel;
    const int L = shard_record_len(k.r);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < k.n; i += (long long)gridDim.x * blockDim.x) {
        const T v = rows_all[i];
        const double lam_g = rec[(size_t)(i / chunk) * L];
        b.logw[i] = (v == T(-INFINITY)) ? T(-INFINITY) : (T)((double)v - (lam - lam_g));
    }
}

template <typename T>
cudaError_t launch_merge(const yy_filter* f, const Consts<T>& k, const Bufs<T>& b, const void* rows_all,
                         const double* rec, int G, cudaStream_t s) {
    const long long chunk = f->n_pad / G;
    k_merge_scalars<T><<<1, 32, 0, s>>>(k, b, rec, G, f->cfg.restart_interval, f->cfg.ess_frac);
    k_merge_dims<T><<<(k.r + 255) / 256, 256, 0, s>>>(k, b, rec, G);
    const unsigned grid = (unsigned)std::min<long long>((k.n + 255) / 256, 1216);
    k_merge_rows<T><<<grid, 256, 0, s>>>(k, b, static_cast<const T*>(rows_all), rec, chunk);
    return cudaGetLastError();
}

}  // namespace

}  // namespace yy

using namespace yy;

extern "C" {

yy_status yy_set_shard(yy_filter* f, int32_t rank, int32_t count) {
    if (!f || count < 1 || count > kMaxShards || rank < 0 || rank >= count) return YY_ERR_ARG;
    if (f->n_pad % (256LL * count) != 0) return YY_ERR_ARG;   // equal chunks of whole 256-row tiles
    if (f->predicted || f->shard_updated) return YY_ERR_STATE;
    const long long chunk = f->n_pad / count;
    f->shard_rank = rank;
    f->shard_count = count;
    f->row0 = std::min<long long>(f->cfg.n, (long long)rank * chunk);
    f->row1 = std::min<long long>(f->cfg.n, (long long)(rank + 1) * chunk);
    f->kf.row0 = f->kd.row0 = f->row0;
    f->kf.row1 = f->kd.row1 = f->row1;
    // a shard screens its own target tiles against every source tile (the symmetric screen
    // would add terms to other shards' rows)
    f->kf.tc_sym = (count == 1 && f->cfg.precision == YY_PREC_BF16 && f->cfg.r > 64) ? 1 : 0;
    if (f->nodes_ready && f->cfg.precision == YY_PREC_BF16) return rebuild_tc_schedule(f);
    return YY_OK;
}

yy_status yy_shard_rows(const yy_filter* f, int64_t* h_row0, int64_t* h_chunk) {
    if (!f) return YY_ERR_ARG;
    if (h_row0) *h_row0 = (int64_t)f->shard_rank * (f->n_pad / f->shard_count);
    if (h_chunk) *h_chunk = f->n_pad / f->shard_count;
    return YY_OK;
}

yy_status yy_update_shard(yy_filter* f, const double* d_dy, void* d_rows_out, double* d_record_out) {
    if (!f || !d_dy || !d_rows_out || !d_record_out) return YY_ERR_ARG;
    if (!f->nodes_ready || !f->predicted || f->shard_updated) return YY_ERR_STATE;
    int l = 0;
    const long long chunk = f->n_pad / f->shard_count;
    const long long first = (long long)f->shard_rank * chunk;
    cudaError_t e;
    if (f->fp64) {
        e = launch_update_shard<double>(f->kd, f->bd, d_dy, d_record_out, f->stream, &l);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_rows_out, f->bd.logw + first, sizeof(double) * chunk, cudaMemcpyDeviceToDevice,
                                f->stream);
    } else {
        e = launch_update_shard<float>(f->kf, f->bf, d_dy, d_record_out, f->stream, &l);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_rows_out, f->bf.logw + first, sizeof(float) * chunk, cudaMemcpyDeviceToDevice,
                                f->stream);
    }
    f->launches += l;
    if (e != cudaSuccess) return YY_ERR_CUDA;
    f->predicted = false;
    f->shard_updated = true;
    return YY_OK;
}

yy_status yy_merge_shards(yy_filter* f, const void* d_rows_all, const double* d_records, int32_t count) {
    if (!f || !d_rows_all || !d_records) return YY_ERR_ARG;
    if (count != f->shard_count) return YY_ERR_ARG;
    if (!f->shard_updated) return YY_ERR_STATE;
    const cudaError_t e = f->fp64 ? launch_merge<double>(f, f->kd, f->bd, d_rows_all, d_records, count, f->stream)
                                  : launch_merge<float>(f, f->kf, f->bf, d_rows_all, d_records, count, f->stream);
    f->launches += 3;
    if (e != cudaSuccess) return YY_ERR_CUDA;
    f->shard_updated = false;
    return YY_OK;
}

yy_status yy_merge_records_host(const double* h_records, int32_t count, int32_t r, double* h_out) {
    if (!h_records || !h_out || count < 1 || count > kMaxShards || r < 1 || r > YY_MAX_DIM) return YY_ERR_ARG;
    double s[kMaxShards];
    double lam, W, Q;
    shard_merge_scalars(h_records, count, r, &lam, &W, &Q, s);
    h_out[0] = lam;
    h_out[1] = W;
    h_out[2] = Q;
    h_out[3] = (Q > 0.0) ? W * W / Q : 0.0;
    for (int d = 0; d < r; ++d) {
        double mu, m2;
        shard_merge_dim(h_records, count, r, s, d, &mu, &m2);
        h_out[4 + d] = mu;
        h_out[4 + r + d] = (W > 0.0) ? m2 / W : 0.0;
    }
    return YY_OK;
}

}  // extern "C"
