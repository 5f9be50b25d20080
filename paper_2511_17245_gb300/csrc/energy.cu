// energy.cu -- E(z) of Eq. def_HUIO for a batch of states, and the sweep
// dispatcher.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sa_internal.h"

namespace sa {

int launch_sweep_quio_i64(const SweepArgs&, int, int, bool, int, int, size_t, void*);
int launch_sweep_quio_f32(const SweepArgs&, int, int, bool, int, int, size_t, void*);
int launch_sweep_huio_i64(const SweepArgs&, int, int, bool, int, int, size_t, void*);
int launch_sweep_huio_f32(const SweepArgs&, int, int, bool, int, int, size_t, void*);

int launch_sweep(const SweepArgs& a, int zbytes, int rule, bool smem, int blocks, int threads, size_t shared_bytes,
                 void* stream) {
    if (a.m.kind == KIND_QUIO) {
        if (a.m.is_float) return launch_sweep_quio_f32(a, zbytes, rule, smem, blocks, threads, shared_bytes, stream);
        return launch_sweep_quio_i64(a, zbytes, rule, smem, blocks, threads, shared_bytes, stream);
    }
    if (a.m.is_float) return launch_sweep_huio_f32(a, zbytes, rule, smem, blocks, threads, shared_bytes, stream);
    return launch_sweep_huio_i64(a, zbytes, rule, smem, blocks, threads, shared_bytes, stream);
}

int launch_sliced_quio_i64(const SweepArgs&, int, int, int, int, size_t, void*, int*);
int launch_sliced_quio_f32(const SweepArgs&, int, int, int, int, size_t, void*, int*);
int launch_sliced_huio_i64(const SweepArgs&, int, int, int, int, size_t, void*, int*);
int launch_sliced_huio_f32(const SweepArgs&, int, int, int, int, size_t, void*, int*);

int launch_sweep_sliced(const SweepArgs& a, int zbytes, int rule, int grid, int threads, size_t shared_bytes,
                        void* stream, int* bps) {
    if (a.m.kind == KIND_QUIO) {
        if (a.m.is_float) return launch_sliced_quio_f32(a, zbytes, rule, grid, threads, shared_bytes, stream, bps);
        return launch_sliced_quio_i64(a, zbytes, rule, grid, threads, shared_bytes, stream, bps);
    }
    if (a.m.is_float) return launch_sliced_huio_f32(a, zbytes, rule, grid, threads, shared_bytes, stream, bps);
    return launch_sliced_huio_i64(a, zbytes, rule, grid, threads, shared_bytes, stream, bps);
}

int launch_batch_quio_i64(const BatchArgs&, int, int, bool, int, int, size_t, void*, bool);
int launch_batch_quio_f32(const BatchArgs&, int, int, bool, int, int, size_t, void*, bool);
int launch_batch_huio_i64(const BatchArgs&, int, int, bool, int, int, size_t, void*, bool);
int launch_batch_huio_f32(const BatchArgs&, int, int, bool, int, int, size_t, void*, bool);

int launch_batch(const BatchArgs& b, int is_float, int kind, int zbytes, int rule, bool smem, int blocks, int threads,
                 size_t shared_bytes, void* stream, bool set_attr) {
    if (kind == KIND_QUIO) {
        if (is_float) return launch_batch_quio_f32(b, zbytes, rule, smem, blocks, threads, shared_bytes, stream, set_attr);
        return launch_batch_quio_i64(b, zbytes, rule, smem, blocks, threads, shared_bytes, stream, set_attr);
    }
    if (is_float) return launch_batch_huio_f32(b, zbytes, rule, smem, blocks, threads, shared_bytes, stream, set_attr);
    return launch_batch_huio_i64(b, zbytes, rule, smem, blocks, threads, shared_bytes, stream, set_attr);
}

int sweep_max_shared_optin() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

namespace {

template <class T>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    T tot = T(0);
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
    return tot;
}

__device__ __forceinline__ long long ipow_ll(long long x, int e) {
    long long r = 1;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}
__device__ __forceinline__ double ipow_d(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

// One block per state.  QUIO: sum_k z_k (lin_k + diag_k z_k) + (1/2) sum over
// the symmetric adjacency.  HUIO: single-variable slots + interaction terms.
template <bool IS_FLOAT>
__global__ void __launch_bounds__(256) energy_kernel(const EnergyArgs a) {
    __shared__ long long red_i[8];
    __shared__ double red_d[8];
    const DevModel& m = a.m;
    const int64_t st = blockIdx.x;
    if (st >= a.n_states) return;
    const int32_t* z = a.states + st * (int64_t)m.n;
    long long e_i = 0, p_i = 0;
    double e_d = 0.0, p_d = 0.0;
    // bounds check: a value outside [l_k, u_k] is reported and not evaluated
    for (int k = threadIdx.x; k < m.n; k += blockDim.x) {
        const VarMeta mt = m.meta[k];
        const long long zk = z[k];
        if (zk < mt.lo || zk > (long long)mt.lo + (long long)mt.width) atomicExch(a.bad, 1);
    }
    if (m.kind == KIND_QUIO) {
        for (int k = threadIdx.x; k < m.n; k += blockDim.x) {
            const VarMeta mt = m.meta[k];
            long long zk = z[k];
            if (zk < mt.lo || zk > (long long)mt.lo + (long long)mt.width) continue;
            if (IS_FLOAT) {
                double f = 0.0;
                for (int e = mt.link_begin; e < mt.link_begin + mt.link_len; ++e)
                    f += (m.adj_d ? m.adj_d[e] : (double)m.adj_f[e]) * (double)z[m.adj_col[e]];
                e_d += (double)zk * (m.lin_d[k] + m.diag_d[k] * (double)zk);
                p_d += (double)zk * f;
            } else {
                long long f = 0;
                for (int e = mt.link_begin; e < mt.link_begin + mt.link_len; ++e) f += m.adj_i[e] * (long long)z[m.adj_col[e]];
                e_i += zk * (m.lin_i[k] + m.diag_i[k] * zk);
                p_i += zk * f;
            }
        }
    } else {
        for (int k = threadIdx.x; k < m.n; k += blockDim.x) {
            const VarMeta mt = m.meta[k];
            const long long zk = z[k];
            if (zk < mt.lo || zk > (long long)mt.lo + (long long)mt.width) continue;
            const int base = m.slot_base[k];
            uint64_t msk = m.omega[k] >> 1;
            int q = 0;
            long long pz = 1;
            double pzd = 1.0;
            while (msk) {
                pz *= zk;
                pzd *= (double)zk;
                if (msk & 1ull) {
                    if (IS_FLOAT) e_d += m.aconst_d[base + q] * pzd;
                    else e_i += m.aconst_i[base + q] * pz;
                    ++q;
                }
                msk >>= 1;
            }
        }
        for (int t = threadIdx.x; t < m.n_iterms; t += blockDim.x) {
            bool inb = true;
            if (IS_FLOAT) {
                double prod = m.tcoef_d[t];
                for (int p = m.term_ptr[t]; p < m.term_ptr[t + 1]; ++p) {
                    const int v = m.mem_var[p];
                    const VarMeta mv = m.meta[v];
                    if (z[v] < mv.lo || (long long)z[v] > (long long)mv.lo + (long long)mv.width) inb = false;
                    prod *= ipow_d((double)z[v], m.mem_exp[p]);
                }
                if (inb) e_d += prod;
            } else {
                long long prod = m.tcoef_i[t];
                for (int p = m.term_ptr[t]; p < m.term_ptr[t + 1]; ++p) {
                    const int v = m.mem_var[p];
                    const VarMeta mv = m.meta[v];
                    if (z[v] < mv.lo || (long long)z[v] > (long long)mv.lo + (long long)mv.width) inb = false;
                    prod *= ipow_ll((long long)z[v], m.mem_exp[p]);
                }
                if (inb) e_i += prod;
            }
        }
    }
    if (IS_FLOAT) {
        const double a1 = block_sum<double>(e_d, red_d);
        __syncthreads();
        const double a2 = block_sum<double>(p_d, red_d);
        if (threadIdx.x == 0) reinterpret_cast<double*>(a.energies)[st] = m.const_d + a1 + 0.5 * a2;
    } else {
        const long long a1 = block_sum<long long>(e_i, red_i);
        __syncthreads();
        const long long a2 = block_sum<long long>(p_i, red_i);
        if (threadIdx.x == 0) reinterpret_cast<long long*>(a.energies)[st] = m.const_i + a1 + a2 / 2;
    }
}

}  // namespace

int launch_energy(const EnergyArgs& a, void* stream) {
    if (a.n_states <= 0) return 0;
    const unsigned grid = (unsigned)a.n_states;
    if (a.m.is_float) energy_kernel<true><<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    else energy_kernel<false><<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace sa
