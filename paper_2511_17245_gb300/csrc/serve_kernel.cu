// serve_kernel.cu -- the persistent kernel behind the request server
// (server.cu): every thread group repeatedly claims the next (request,
// replica) unit of a work queue that the host keeps appending to, copies the
// request's run arguments into shared memory and runs that replica with the
// sweep code of sa_run (same random numbers, so a replica's result does not
// depend on what else is queued).  Requests of every rule, model kind,
// coefficient class and state width share the queue: each unit dispatches to
// one of 24 compiled variants, each kept out of line so that it gets the
// register allocation of a stand-alone kernel.
#include <cuda_runtime.h>

#include "sweep.cuh"

namespace sa {
namespace dev {

template <class F, class Z, int RULE, int KIND>
__device__ __noinline__ void serve_body(const SweepArgs& a, int slot, int t, int r, uint8_t* base) {
    replica_body<F, Z, RULE, KIND>(a, slot, t, r, base);
}

template <class F, class Z, int KIND>
__device__ __forceinline__ void serve_rule(int rule, const SweepArgs& a, int slot, int t, int r, uint8_t* base) {
    if (rule == RULE_METROPOLIS) serve_body<F, Z, RULE_METROPOLIS, KIND>(a, slot, t, r, base);
    else if (rule == RULE_HEAT_BATH) serve_body<F, Z, RULE_HEAT_BATH, KIND>(a, slot, t, r, base);
    else serve_body<F, Z, RULE_OPT, KIND>(a, slot, t, r, base);
}

template <class Z>
__device__ __forceinline__ void serve_dispatch(int v, const SweepArgs& a, int slot, int t, int r, uint8_t* base) {
    const int rule = v % 3, kind = (v / 3) % 2, is_float = (v / 6) % 2;
    if (is_float) {
        if (kind == KIND_QUIO) serve_rule<float, Z, KIND_QUIO>(rule, a, slot, t, r, base);
        else serve_rule<float, Z, KIND_HUIO>(rule, a, slot, t, r, base);
    } else {
        if (kind == KIND_QUIO) serve_rule<long long, Z, KIND_QUIO>(rule, a, slot, t, r, base);
        else serve_rule<long long, Z, KIND_HUIO>(rule, a, slot, t, r, base);
    }
}

__device__ __forceinline__ unsigned int ld_acquire_sys(const volatile unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys(unsigned int* p, unsigned int v) {
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr int kServeMaxGroups = 8;

__global__ void __launch_bounds__(512, 1) serve_kernel(const ServeArgs s) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ __align__(16) SweepArgs args_s[kServeMaxGroups];
    __shared__ int unit_s[kServeMaxGroups][3];
    const int slot = threadIdx.x / s.tpr;
    const int t = threadIdx.x - slot * s.tpr;
    if (slot >= s.rpc || slot >= kServeMaxGroups) return;
    const int bar_id = 1 + slot;
    for (;;) {
        if (t == 0) {
            // claim the next published unit; an empty queue is polled (bounded)
            int req = -1, rep = 0, variant = 0;
            for (uint32_t idle = 0;;) {
                const unsigned int tail = ld_acquire_sys(&s.ctl->tail);
                const unsigned int h = *reinterpret_cast<volatile unsigned int*>(s.head);
                if (h < tail) {
                    if (atomicCAS(s.head, h, h + 1u) == h) {
                        const volatile ServeUnit* u = s.units + (h & (s.cap - 1u));
                        req = u->req;
                        rep = u->replica;
                        variant = reinterpret_cast<const volatile ServeReq*>(s.reqs + req)->variant;
                        break;
                    }
                    continue;
                }
                if (*reinterpret_cast<const volatile unsigned int*>(&s.ctl->stop) != 0u || ++idle > s.idle_polls) break;
                __nanosleep(2000);
            }
            unit_s[slot][0] = req;
            unit_s[slot][1] = rep;
            unit_s[slot][2] = variant;
        }
        named_bar(bar_id, s.tpr);
        const int req = unit_s[slot][0];
        if (req < 0) break;
        const int rep = unit_s[slot][1], variant = unit_s[slot][2];
        {
            const volatile uint32_t* src = reinterpret_cast<const volatile uint32_t*>(&s.reqs[req].args);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&args_s[slot]);
            for (int w = t; w < (int)(sizeof(SweepArgs) / 4); w += s.tpr) dst[w] = src[w];
        }
        named_bar(bar_id, s.tpr);
        const SweepArgs& a = args_s[slot];
        // replica state: the group's shared-memory region when it fits, else
        // the request's slab in global memory
        uint8_t* base = a.gstate != nullptr ? a.gstate + (size_t)rep * (size_t)a.rep_bytes
                                            : smem_raw + (size_t)slot * (size_t)s.slot_bytes;
        if (variant >= 12) serve_dispatch<uint32_t>(variant - 12, a, slot, t, rep, base);
        else serve_dispatch<uint16_t>(variant, a, slot, t, rep, base);
        __threadfence();                 // this thread's outputs before the unit counts as done
        named_bar(bar_id, s.tpr);        // the group is done with args_s, unit_s and the region
        if (t == 0) {
            const unsigned int done = atomicAdd(s.req_units_done + req, 1u) + 1u;
            if (done == (unsigned int)reinterpret_cast<const volatile ServeReq*>(s.reqs + req)->n_units) {
                __threadfence_system();
                st_release_sys(s.req_done + req, 1u);
            }
        }
    }
}

}  // namespace dev

int launch_serve(const ServeArgs& s, int grid, size_t shared_bytes, void* stream) {
    auto kern = dev::serve_kernel;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shared_bytes);
    if (e != cudaSuccess || grid == 0) return (int)e;
    kern<<<grid, s.rpc * s.tpr, shared_bytes, (cudaStream_t)stream>>>(s);
    return (int)cudaGetLastError();
}

size_t serve_static_shared() { return sizeof(SweepArgs) * dev::kServeMaxGroups + 16 * dev::kServeMaxGroups + 64; }

}  // namespace sa
