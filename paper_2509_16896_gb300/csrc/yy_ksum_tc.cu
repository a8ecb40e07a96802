// Prediction step, BF16 tensor-core screening + exact float32 evaluation (placeholder).
#include "yy_internal.cuh"

namespace yy {

size_t tc_scratch_bytes(long long n_pad, int N) {
    return 256 + (size_t)n_pad * 2 * N * sizeof(float) + 256 + (size_t)n_pad * 16 * sizeof(int2);
}

cudaError_t launch_ksum_tc(const Consts<float>&, const Bufs<float>&, cudaStream_t, int*) {
    return cudaErrorNotSupported;
}

}  // namespace yy
