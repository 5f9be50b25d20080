// sweep_launch.cuh -- instantiates the sweep kernel for one (field type,
// model kind) pair over z width, rule and state placement.
#pragma once

#include "sweep.cuh"

namespace sa {

template <class F, class Z, int RULE, int KIND, bool SMEM>
static int launch_one(const SweepArgs& a, int blocks, int threads, size_t shared_bytes, cudaStream_t st) {
    auto kern = dev::sweep_kernel<F, Z, RULE, KIND, SMEM>;
    if (shared_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shared_bytes);
        if (e != cudaSuccess) return (int)e;
    }
    kern<<<blocks, threads, shared_bytes, st>>>(a);
    return (int)cudaGetLastError();
}

template <class F, class Z, int KIND, bool SMEM>
static int launch_rule(const SweepArgs& a, int rule, int blocks, int threads, size_t sh, cudaStream_t st) {
    switch (rule) {
    case RULE_METROPOLIS: return launch_one<F, Z, RULE_METROPOLIS, KIND, SMEM>(a, blocks, threads, sh, st);
    case RULE_HEAT_BATH: return launch_one<F, Z, RULE_HEAT_BATH, KIND, SMEM>(a, blocks, threads, sh, st);
    default: return launch_one<F, Z, RULE_OPT, KIND, SMEM>(a, blocks, threads, sh, st);
    }
}

template <class F, int KIND>
static int launch_family(const SweepArgs& a, int zbytes, int rule, bool smem, int blocks, int threads,
                         size_t sh, cudaStream_t st) {
    if (smem) {
        if (zbytes == 1) return launch_rule<F, uint8_t, KIND, true>(a, rule, blocks, threads, sh, st);
        if (zbytes == 2) return launch_rule<F, uint16_t, KIND, true>(a, rule, blocks, threads, sh, st);
        return launch_rule<F, uint32_t, KIND, true>(a, rule, blocks, threads, sh, st);
    }
    if (zbytes == 1) return launch_rule<F, uint8_t, KIND, false>(a, rule, blocks, threads, sh, st);
    if (zbytes == 2) return launch_rule<F, uint16_t, KIND, false>(a, rule, blocks, threads, sh, st);
    return launch_rule<F, uint32_t, KIND, false>(a, rule, blocks, threads, sh, st);
}

template <class F, class Z, int RULE, int KIND>
static int launch_sliced_one(const SweepArgs& a, int grid, int threads, size_t shared_bytes, cudaStream_t st,
                             int* blocks_per_sm) {
    auto kern = dev::sweep_sliced_kernel<F, Z, RULE, KIND>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shared_bytes);
    if (e != cudaSuccess) return (int)e;
    if (grid == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, threads, shared_bytes);
        return (int)e;
    }
    SweepArgs args = a;
    void* params[] = {&args};
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(threads), params, shared_bytes, st);
    return (int)e;
}

template <class F, class Z, int KIND>
static int launch_sliced_rule(const SweepArgs& a, int rule, int grid, int threads, size_t sh, cudaStream_t st,
                              int* bps) {
    switch (rule) {
    case RULE_METROPOLIS: return launch_sliced_one<F, Z, RULE_METROPOLIS, KIND>(a, grid, threads, sh, st, bps);
    case RULE_HEAT_BATH: return launch_sliced_one<F, Z, RULE_HEAT_BATH, KIND>(a, grid, threads, sh, st, bps);
    default: return launch_sliced_one<F, Z, RULE_OPT, KIND>(a, grid, threads, sh, st, bps);
    }
}

template <class F, int KIND>
static int launch_sliced_family(const SweepArgs& a, int zbytes, int rule, int grid, int threads, size_t sh,
                                cudaStream_t st, int* bps) {
    if (zbytes == 1) return launch_sliced_rule<F, uint8_t, KIND>(a, rule, grid, threads, sh, st, bps);
    if (zbytes == 2) return launch_sliced_rule<F, uint16_t, KIND>(a, rule, grid, threads, sh, st, bps);
    return launch_sliced_rule<F, uint32_t, KIND>(a, rule, grid, threads, sh, st, bps);
}

template <class F, class Z, int RULE, int KIND, bool SMEM>
static int launch_batch_one(const BatchArgs& b, int blocks, int threads, size_t shared_bytes, cudaStream_t st,
                            bool set_attr) {
    auto kern = dev::batch_kernel<F, Z, RULE, KIND, SMEM>;
    if (set_attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shared_bytes);
        if (e != cudaSuccess) return (int)e;
    }
    if (blocks == 0) return 0;   // attribute only (before a stream capture)
    kern<<<blocks, threads, shared_bytes, st>>>(b);
    return (int)cudaGetLastError();
}

template <class F, class Z, int KIND, bool SMEM>
static int launch_batch_rule(const BatchArgs& b, int rule, int blocks, int threads, size_t sh, cudaStream_t st,
                             bool set_attr) {
    switch (rule) {
    case RULE_METROPOLIS: return launch_batch_one<F, Z, RULE_METROPOLIS, KIND, SMEM>(b, blocks, threads, sh, st, set_attr);
    case RULE_HEAT_BATH: return launch_batch_one<F, Z, RULE_HEAT_BATH, KIND, SMEM>(b, blocks, threads, sh, st, set_attr);
    default: return launch_batch_one<F, Z, RULE_OPT, KIND, SMEM>(b, blocks, threads, sh, st, set_attr);
    }
}

template <class F, int KIND>
static int launch_batch_family(const BatchArgs& b, int zbytes, int rule, bool smem, int blocks, int threads,
                               size_t sh, cudaStream_t st, bool set_attr) {
    if (smem) {
        if (zbytes == 1) return launch_batch_rule<F, uint8_t, KIND, true>(b, rule, blocks, threads, sh, st, set_attr);
        if (zbytes == 2) return launch_batch_rule<F, uint16_t, KIND, true>(b, rule, blocks, threads, sh, st, set_attr);
        return launch_batch_rule<F, uint32_t, KIND, true>(b, rule, blocks, threads, sh, st, set_attr);
    }
    if (zbytes == 1) return launch_batch_rule<F, uint8_t, KIND, false>(b, rule, blocks, threads, sh, st, set_attr);
    if (zbytes == 2) return launch_batch_rule<F, uint16_t, KIND, false>(b, rule, blocks, threads, sh, st, set_attr);
    return launch_batch_rule<F, uint32_t, KIND, false>(b, rule, blocks, threads, sh, st, set_attr);
}

}  // namespace sa
