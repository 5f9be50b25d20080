// sweep_huio_f32.cu -- sweep kernels for HUIO models with f32 fields.
#include "sweep_launch.cuh"

namespace sa {
int launch_sweep_huio_f32(const SweepArgs& a, int zbytes, int rule, bool smem, int blocks, int threads,
                              size_t sh, void* stream) {
    return launch_family<float, KIND_HUIO>(a, zbytes, rule, smem, blocks, threads, sh, (cudaStream_t)stream);
}
int launch_batch_huio_f32(const BatchArgs& b, int zbytes, int rule, bool smem, int blocks, int threads,
                             size_t sh, void* stream, bool set_attr) {
    return launch_batch_family<float, KIND_HUIO>(b, zbytes, rule, smem, blocks, threads, sh, (cudaStream_t)stream, set_attr);
}
int launch_sliced_huio_f32(const SweepArgs& a, int zbytes, int rule, int grid, int threads, size_t sh, void* stream,
                        int* bps) {
    return launch_sliced_family<float, KIND_HUIO>(a, zbytes, rule, grid, threads, sh, (cudaStream_t)stream, bps);
}
}  // namespace sa
