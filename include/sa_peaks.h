/*
 * sa_peaks.h -- measured throughput ceilings of the current GPU, for the
 * roofline fractions the benchmark reports next to the sweep kernels.
 *
 * The paper has no counterpart: this is a measurement service of the library,
 * not a step of the method.  The sweep kernels keep their state in shared
 * memory, read the model through L2 and spend their arithmetic on fp32 FMAs
 * and (heat bath) exp2 evaluations, so the relevant ceilings are those of the
 * SFU, the FMA pipe, L2 and shared memory rather than HBM alone.
 */
#ifndef SA_GB300_PEAKS_H
#define SA_GB300_PEAKS_H

#include <stdint.h>

#include "sa.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double exp2_per_s;         /* ex2.approx.ftz.f32 results per second (SFU)            */
    double fma_per_s;          /* fp32 FMA results per second                             */
    double l2_gbs;             /* copy of an L2-resident buffer: bytes read + written / s */
    double smem_gbs;           /* shared memory: 16-byte loads + stores, bytes / s        */
    double smem_atomic_per_s;  /* fp32 atomicAdd on distinct shared-memory words / s      */
    int32_t sms;               /* streaming multiprocessors of the device                 */
    int32_t l2_buffer_bytes;   /* size of the copied buffer (source + destination)        */
    float exp2_ms, fma_ms, l2_ms, smem_ms, smem_atomic_ms;   /* timed launch durations   */
} sa_peaks;

/*
 * sa_measure_peaks -- runs five micro-kernels on `stream` (each once to warm
 * up, then timed with CUDA events, best of three) on the current device and
 * fills `out`.  Every kernel keeps all SMs busy with independent work:
 *   exp2        8 independent chains x <- 2^x - 1 per thread (x stays in
 *               [-0.3, 0]), 64 warps per SM;
 *   fma         8 independent chains x <- x * a + b per thread;
 *   l2          float4 copy of a buffer that fits in L2 (loads and stores
 *               marked cache-global), repeated passes;
 *   smem        float4 loads and stores of distinct, conflict-free words;
 *   smem_atomic fp32 atomicAdd on distinct shared words, 32 per warp.
 * Allocates (and frees) the L2 buffers with cudaMalloc; synchronises `stream`.
 * Errors: SA_ERR_INVALID for a NULL `out`, SA_ERR_OOM / SA_ERR_CUDA for device
 * failures (message in sa_last_error()).
 */
sa_status sa_measure_peaks(sa_peaks* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SA_GB300_PEAKS_H */
