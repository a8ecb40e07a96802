// Host-side handle of one filter (shared by the single-filter and batch entry points).
#pragma once

#include "yy_internal.cuh"

struct yy_filter {
    yy_config cfg;
    int r_pad;
    long long n_pad;
    cudaStream_t stream;
    char* ws;
    size_t ws_bytes;
    bool fp64;
    yy::Bufs<float> bf;
    yy::Bufs<double> bd;
    yy::Consts<float> kf;
    yy::Consts<double> kd;
    bool nodes_ready;
    bool predicted;     // logw_pred holds the last prediction
    long long launches;
    double coef[yy::kMaxScales + 1];
    double log_wq;
    double c_ref;
    cudaGraph_t graph;
    cudaGraphExec_t gexec;
    long long graph_kernels;
    struct yy_mlp* mlp;   // restart-proposal network for YY_RESTART_LEARNED (not owned)
    unsigned long long wait_ns;   // limit of bounded device waits (default 4 s)
    long long row0, row1;         // target rows of this handle (shards of a row-split filter)
    int shard_rank, shard_count;  // 0, 1 for a whole filter
    bool shard_updated;           // yy_update_shard ran; yy_merge_shards completes the step
    int node_kind;                // yy_nodes of the last node generation
    bool use_op;                  // the prediction applies the materialised operator
    bool pair_ok;                 // the tensor-core prediction may run on CTA pairs (yy_set_cta_pair)
    bool route_plain = false;   // BF16: predictions on the plain float32 form (yy_set_route)
};

namespace yy {
// Rebuilds the work list of the tensor-core prediction for the handle's target rows.
yy_status rebuild_tc_schedule(yy_filter* f);
}  // namespace yy
