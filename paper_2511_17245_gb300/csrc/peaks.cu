// peaks.cu -- micro-kernels that measure the throughput ceilings used as
// roofline denominators (sa_measure_peaks in include/sa_peaks.h).  Each kernel
// keeps every SM busy with independent work of one kind and is timed with CUDA
// events on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "sa.h"
#include "sa_peaks.h"

extern "C" void sa_internal_set_error(const char* msg);

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- 2^x - 1 keeps x in [-0.3, 0]: eight dependent chains per thread.
__global__ void __launch_bounds__(kThreads) exp2_kernel(float* sink, int iters) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = -0.25f * (float)((threadIdx.x + 31 * j) & 63) * (1.0f / 64.0f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = ex2_approx(x[j]) - 1.0f;
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// x <- x a + b: eight dependent FMA chains per thread.
__global__ void __launch_bounds__(kThreads) fma_kernel(float* sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = (float)((threadIdx.x + 7 * j) & 15);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Ping-pong copy between two L2-resident buffers; every element is read and
// written by the same thread in every pass, so passes do not race.  Loads and
// stores are cache-global (L2, not L1).
__global__ void __launch_bounds__(kThreads) l2_copy_kernel(float4* b0, float4* b1, int n4, int passes) {
    const int stride = gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        const float4* src = (p & 1) ? b1 : b0;
        float4* dst = (p & 1) ? b0 : b1;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) __stcg(dst + i, __ldcg(src + i));
    }
}

__device__ __forceinline__ float4 lds128(const float4* p) {
    float4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts128(float4* p, float4 v) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// Thread t owns the 16-byte words t + 256 j (j = 0..3): consecutive threads
// touch consecutive words (no bank conflicts) and no word is shared.  16 KB per
// block, so that the 8 blocks of an SM fit at once.
__global__ void __launch_bounds__(kThreads) smem_kernel(float* sink, int iters) {
    __shared__ float4 buf[4 * kThreads];
    const int t = threadIdx.x;
#pragma unroll
    for (int j = 0; j < 4; ++j) buf[t + kThreads * j] = make_float4((float)j, 0.f, 0.f, 0.f);
    float acc = 0.f;
    for (int it = 0; it < iters; ++it) {
        const int j = it & 3;
        const float4 v0 = lds128(buf + t + kThreads * j);
        const float4 v1 = lds128(buf + t + kThreads * ((j + 1) & 3));
        sts128(buf + t + kThreads * ((j + 2) & 3), v0);
        sts128(buf + t + kThreads * ((j + 3) & 3), v1);
        acc += v0.x;
    }
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// fp32 atomicAdd without a returned value on distinct shared words: a warp's
// 32 lanes hit 32 consecutive words (32 banks).  16 KB per block.
__global__ void __launch_bounds__(kThreads) smem_atomic_kernel(float* sink, int iters) {
    __shared__ float buf[16 * kThreads];
    const int t = threadIdx.x;
    for (int i = t; i < 16 * kThreads; i += kThreads) buf[i] = 0.f;
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) atomicAdd(buf + t + kThreads * ((it * 8 + j) & 15), 1.0f);
    }
    __syncthreads();
    sink[blockIdx.x * blockDim.x + t] = buf[t];
}

struct Timer {
    cudaStream_t st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    explicit Timer(cudaStream_t s) : st(s) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    ~Timer() {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    // best of three timed launches after one warm-up launch; < 0 on error
    template <class F>
    float best(F launch) {
        launch();
        float b = -1.f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            b = (b < 0.f || ms < b) ? ms : b;
        }
        return cudaGetLastError() == cudaSuccess ? b : -1.f;
    }
};

sa_status pfail(sa_status st, const std::string& msg) {
    sa_internal_set_error(msg.c_str());
    return st;
}

}  // namespace

extern "C" sa_status sa_measure_peaks(sa_peaks* out, void* stream) {
    if (!out) return pfail(SA_ERR_INVALID, "out is NULL");
    *out = sa_peaks{};
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) return pfail(SA_ERR_CUDA, "no device");
    out->sms = sms;
    const int blocks = sms * 8;                 // 64 warps per SM
    float* sink = nullptr;
    const int n4 = (16 << 20) / 16;             // 16 MiB per buffer, 32 MiB in L2
    float4* buf = nullptr;
    cudaError_t e = cudaMalloc(&sink, (size_t)blocks * kThreads * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&buf, 2 * (size_t)n4 * sizeof(float4));
    if (e != cudaSuccess) {
        cudaFree(sink);
        return pfail(e == cudaErrorMemoryAllocation ? SA_ERR_OOM : SA_ERR_CUDA,
                     std::string("sa_measure_peaks: ") + cudaGetErrorString(e));
    }
    cudaMemsetAsync(buf, 0, 2 * (size_t)n4 * sizeof(float4), st);
    Timer tm(st);
    const int it_exp = 4096, it_fma = 16384, passes = 256, it_smem = 16384, it_atom = 4096;
    out->exp2_ms = tm.best([&] { exp2_kernel<<<blocks, kThreads, 0, st>>>(sink, it_exp); });
    out->fma_ms = tm.best([&] { fma_kernel<<<blocks, kThreads, 0, st>>>(sink, it_fma, 0.999f, 1e-4f); });
    out->l2_ms = tm.best([&] { l2_copy_kernel<<<sms * 4, kThreads, 0, st>>>(buf, buf + n4, n4, passes); });
    out->smem_ms = tm.best([&] { smem_kernel<<<blocks, kThreads, 0, st>>>(sink, it_smem); });
    out->smem_atomic_ms = tm.best([&] { smem_atomic_kernel<<<blocks, kThreads, 0, st>>>(sink, it_atom); });
    cudaFree(buf);
    cudaFree(sink);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pfail(SA_ERR_CUDA, std::string("sa_measure_peaks: ") + cudaGetErrorString(e));
    if (out->exp2_ms <= 0.f || out->fma_ms <= 0.f || out->l2_ms <= 0.f || out->smem_ms <= 0.f ||
        out->smem_atomic_ms <= 0.f)
        return pfail(SA_ERR_CUDA, "sa_measure_peaks: a timing launch failed");
    const double thr = (double)blocks * kThreads;
    out->exp2_per_s = thr * it_exp * kChains / (out->exp2_ms * 1e-3);
    out->fma_per_s = thr * it_fma * kChains / (out->fma_ms * 1e-3);
    out->l2_buffer_bytes = (int32_t)(2 * (size_t)n4 * sizeof(float4));
    out->l2_gbs = 2.0 * (double)n4 * sizeof(float4) * passes / (out->l2_ms * 1e-3) / 1e9;
    out->smem_gbs = thr * it_smem * 4.0 * 16.0 / (out->smem_ms * 1e-3) / 1e9;
    out->smem_atomic_per_s = thr * it_atom * 8.0 / (out->smem_atomic_ms * 1e-3);
    return SA_OK;
}
