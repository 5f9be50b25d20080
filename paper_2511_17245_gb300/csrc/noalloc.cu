// noalloc.cu -- sa_run_noalloc: the SA run of sa_run for callers that cannot
// allocate device memory.
//
// Some callers are not allowed to call cudaMalloc/cudaFree (or anything that
// allocates on their behalf): a host framework that owns all device memory
// through its own arena and forbids other allocations, or a latency-critical
// service where an allocation (which may synchronise the device) must not
// happen on the request path.  This entry point serves them: the caller passes
// device buffers for every input and output, and the run's own scratch (the
// per-sweep temperature table and, when a replica's state does not fit on
// chip, its state slab) lives in one fixed, file-scope device array of
// SA_NOALLOC_SCRATCH_BYTES bytes that every device loading this library holds
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "sa.h"
#include "sa_internal.h"

extern "C" int sa_internal_model_view(const sa_model* M, sa::ModelView* v);
extern "C" void sa_internal_set_error(const char* msg);

namespace {

// The shared scratch.  Every call on a device uses this same array and it
// keeps whatever the last call left in it; calls whose work overlaps on the
// GPU (two streams, or a second call before the first finished) race on it.
static __device__ __align__(256) unsigned char g_scratch[SA_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

sa_status fail(sa_status st, const std::string& msg) {
    sa_internal_set_error(msg.c_str());
    return st;
}

// Device address of g_scratch on the current device.  In host code the name
// g_scratch only denotes a host-side stand-in, so the address is looked up once
// per device with that device current and cached.
sa_status scratch_address(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(SA_ERR_UNSUPPORTED, "device index beyond the scratch table");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return fail(SA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return SA_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" sa_status sa_run_noalloc(const sa_model* M, const sa_run_params* p, int32_t* out_states,
                                    void* out_energies, uint64_t* out_accepts, void* stream) {
    sa::ModelView mv;
    if (!M || !p || !sa_internal_model_view(M, &mv)) return fail(SA_ERR_INVALID, "NULL model or params");
    if (!out_states || !out_energies) return fail(SA_ERR_INVALID, "NULL output");
    if (p->rule < 0 || p->rule > 2) return fail(SA_ERR_INVALID, "unknown rule");
    if (p->n_sweeps < 1 || p->n_replicas < 1) return fail(SA_ERR_INVALID, "n_sweeps and n_replicas must be positive");
    if (p->report) return fail(SA_ERR_INVALID, "sa_run_noalloc does not fill a report");
    if (p->best_states || p->best_energies)
        return fail(SA_ERR_UNSUPPORTED, "best-state tracking is not available in sa_run_noalloc");
    if (p->trace && (p->trace_replicas < 0 || p->trace_replicas > p->n_replicas))
        return fail(SA_ERR_INVALID, "trace_replicas out of range");
    if (p->rule == SA_OPT_METROPOLIS && mv.max_exp > 4)
        return fail(SA_ERR_UNSUPPORTED, "optimal-transition Metropolis needs exponents <= 4");
    if (!on_device(out_states) || !on_device(out_energies) || (out_accepts && !on_device(out_accepts)) ||
        (p->init_states && !on_device(p->init_states)))
        return fail(SA_ERR_INVALID, "sa_run_noalloc needs device buffers for every input and output");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != mv.device) return fail(SA_ERR_INVALID, "model belongs to another device");
    unsigned char* scratch = nullptr;
    sa_status st0 = scratch_address(dev, &scratch);
    if (st0 != SA_OK) return st0;
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t S = p->n_sweeps, R = p->n_replicas;

    // temperature table and launch shape: the planner sa_run uses (Sect. 3.1,
    // Sect. 3.3.3), so that both entry points give identical runs
    const size_t tab_bytes = round_up(2 * (size_t)S * sizeof(float), 256);
    if (tab_bytes > (size_t)SA_NOALLOC_SCRATCH_BYTES)
        return fail(SA_ERR_UNSUPPORTED, "n_sweeps too large for the fixed scratch of sa_run_noalloc (limit " +
                                            std::to_string(SA_NOALLOC_SCRATCH_BYTES / 8) + " sweeps)");
    std::vector<float> tab(2 * (size_t)S);
    if (const char* err = sa::plan_schedule(mv.de_max, mv.de_min, S, p->t_max, p->t_min, p->temperatures, tab.data()))
        return fail(SA_ERR_INVALID, err);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sa::RunPlan plan{};
    if (const char* err = sa::plan_run_shape(sa::plan_model(mv), R, p->threads_per_replica, p->replicas_per_block,
                                             (p->flags & SA_FLAG_STATE_IN_GLOBAL) != 0, sms,
                                             sa::sweep_max_shared_optin(), &plan))
        return fail(SA_ERR_INVALID, err);
    const bool in_global = plan.in_global != 0;
    const size_t slab_bytes = in_global ? (size_t)R * (size_t)plan.rep_bytes : 0;
    if (tab_bytes + slab_bytes > (size_t)SA_NOALLOC_SCRATCH_BYTES)
        return fail(SA_ERR_UNSUPPORTED, "replica state does not fit on chip and " + std::to_string(R) +
                                            " replicas exceed the fixed scratch of sa_run_noalloc (" +
                                            std::to_string(SA_NOALLOC_SCRATCH_BYTES) + " bytes)");

    float* d_tab = reinterpret_cast<float*>(scratch);
    cudaError_t e = cudaMemcpyAsync(d_tab, tab.data(), 2 * (size_t)S * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(SA_ERR_CUDA, std::string("copy schedule: ") + cudaGetErrorString(e));

    sa::SweepArgs a{};
    a.m = mv.dm;
    a.R = R;
    a.S = S;
    a.key0 = (uint32_t)(p->seed & 0xFFFFFFFFull);
    a.key1 = (uint32_t)(p->seed >> 32);
    a.inst = p->instance_id;
    a.refresh_interval = p->refresh_interval > 0 ? p->refresh_interval : 50;
    a.speculate = (p->flags & SA_FLAG_NO_SPECULATION) ? 0 : 1;
    a.beta = d_tab;
    a.ratio = d_tab + S;
    a.init_states = p->init_states;
    a.out_states = out_states;
    a.out_energies = out_energies;
    a.out_accepts = (unsigned long long*)out_accepts;
    a.trace = p->trace;
    a.trace_R = p->trace ? p->trace_replicas : 0;
    a.energy_trace = p->energy_trace;
    a.drift_bits = nullptr;
    a.gstate = in_global ? scratch + tab_bytes : nullptr;   // every slab byte is written before it is read
    sa::plan_apply(plan, a);
    const int le = sa::launch_sweep(a, mv.zbytes, p->rule, !in_global, plan.blocks, plan.rpc * plan.tpr,
                                   (size_t)plan.shared_bytes, stream);
    if (le != 0) return fail(SA_ERR_CUDA, std::string("sweep launch: ") + cudaGetErrorString((cudaError_t)le));
    return SA_OK;
}
