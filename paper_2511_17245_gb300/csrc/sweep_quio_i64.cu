// sweep_quio_i64.cu -- sweep kernels for QUIO models with i64 fields.
#include "sweep_launch.cuh"

namespace sa {
int launch_sweep_quio_i64(const SweepArgs& a, int zbytes, int rule, bool smem, int blocks, int threads,
                              size_t sh, void* stream) {
    return launch_family<long long, KIND_QUIO>(a, zbytes, rule, smem, blocks, threads, sh, (cudaStream_t)stream);
}
int launch_batch_quio_i64(const BatchArgs& b, int zbytes, int rule, bool smem, int blocks, int threads,
                             size_t sh, void* stream, bool set_attr) {
    return launch_batch_family<long long, KIND_QUIO>(b, zbytes, rule, smem, blocks, threads, sh, (cudaStream_t)stream, set_attr);
}
int launch_sliced_quio_i64(const SweepArgs& a, int zbytes, int rule, int grid, int threads, size_t sh, void* stream,
                        int* bps) {
    return launch_sliced_family<long long, KIND_QUIO>(a, zbytes, rule, grid, threads, sh, (cudaStream_t)stream, bps);
}
}  // namespace sa
