// batch.cu -- many SA instances in one persistent, CUDA-graph-captured launch.
//
// A batch holds the per-instance kernel arguments, the per-instance schedules
// (Sect. 3.1, Sect. 3.3.3; temperatures from Sect. 3.4 unless given), the
// output buffers and a list of work units (one replica of one instance each)
// ordered by decreasing estimated cost.  The persistent kernel's thread groups
// claim units from a global counter, so uneven instances (sizes, ranges,
// densities) balance across the GPU.  The launch (counter reset + kernel) is
// captured once in a CUDA graph and replayed by sa_batch_run.  The launch
// shape (threads per replica, replicas per block) is chosen by a heuristic or
// by sa_batch_autotune, which times candidate shapes on a truncated run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sa.h"
#include "sa_internal.h"

extern "C" int sa_internal_model_view(const sa_model* M, sa::ModelView* v);
extern "C" void sa_internal_set_error(const char* msg);

namespace {

sa_status bfail(sa_status st, const std::string& msg) {
    sa_internal_set_error(msg.c_str());
    return st;
}
sa_status bcuda(cudaError_t e, const char* where) {
    return bfail(e == cudaErrorMemoryAllocation ? SA_ERR_OOM : SA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
size_t up256(size_t x) { return (x + 255) / 256 * 256; }
bool dev_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct sa_batch {
    int device = 0;
    int n = 0;
    int kind = 0, is_float = 0, zbytes = 1, rule = 0;
    std::vector<sa::ModelView> views;
    std::vector<int32_t> R, S;
    std::vector<int64_t> st_off, en_off;
    std::vector<sa::SweepArgs> h_insts;
    std::vector<sa::BatchUnit> h_units;
    int64_t attempts = 0;
    void* dmem = nullptr;
    size_t dbytes = 0;
    sa::SweepArgs* d_insts = nullptr;
    sa::BatchUnit* d_units = nullptr;
    unsigned int* d_counter = nullptr;
    int32_t* d_states = nullptr;
    void* d_energies = nullptr;
    unsigned long long* d_accepts = nullptr;
    uint8_t* d_gstate = nullptr;
    size_t gstate_bytes = 0;
    int rpc = 0, tpr = 0, blocks = 0;
    size_t slot_bytes = 0;
    bool smem = true;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    float last_ms = 0.f;
};

namespace {

// Per-instance state layout for a given threads-per-replica: the layout of
// sa_run (shared planner) with the batch's widest state offsets.
size_t layout(sa::SweepArgs& a, const sa::ModelView& v, int zb, int tpr) {
    sa::RunPlan pl{};
    const int64_t rep = sa::plan_layout(sa::plan_model(v), zb, tpr, &pl);
    pl.rpc = a.rpc;
    sa::plan_apply(pl, a);
    return (size_t)rep;
}

// Sets the launch shape and rebuilds the per-instance arguments for it.
sa_status apply_shape(sa_batch* b, int tpr, int rpc_req) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    size_t slot = 0;
    for (int i = 0; i < b->n; ++i) slot = std::max(slot, layout(b->h_insts[i], b->views[i], b->zbytes, tpr));
    const int smem_max = sa::sweep_max_shared_optin() - 8192;   // leave room for the static argument copies
    int fit = (int)((size_t)std::max(0, smem_max) / slot);
    fit = std::min(fit, std::min(15, 512 / tpr));
    bool smem = fit >= 1;
    int rpc = rpc_req > 0 ? rpc_req : (smem ? fit : std::min(15, 512 / tpr));
    if (rpc < 1 || rpc > 15 || rpc * tpr > 512) return bfail(SA_ERR_INVALID, "batch launch shape out of range");
    if (smem && rpc > fit) return bfail(SA_ERR_INVALID, "replicas_per_block exceeds shared memory");
    // persistent grid: as many blocks as fit on the GPU at once (1 per SM with large shared use)
    int per_sm = 1;
    if (smem) per_sm = std::max(1, std::min((int)((size_t)sa::sweep_max_shared_optin() / ((size_t)rpc * slot + 8192)),
                                            2048 / (rpc * tpr)));
    else per_sm = std::max(1, 2048 / (rpc * tpr));
    per_sm = std::min(per_sm, std::max(1, 65536 / (rpc * tpr * 128)));   // registers: up to 128 per thread
    int blocks = sms * per_sm;
    const int need = (int)((b->h_units.size() + rpc - 1) / rpc);
    blocks = std::max(1, std::min(blocks, need));
    if (!smem) {
        const size_t gb = (size_t)blocks * rpc * slot;
        if (gb > b->gstate_bytes) {
            if (b->d_gstate) cudaFree(b->d_gstate);
            b->d_gstate = nullptr;
            b->gstate_bytes = 0;
            cudaError_t e = cudaMalloc(&b->d_gstate, gb);
            if (e != cudaSuccess) return bcuda(e, "cudaMalloc(batch state)");
            b->gstate_bytes = gb;
        }
    }
    b->tpr = tpr;
    b->rpc = rpc;
    b->blocks = blocks;
    b->slot_bytes = slot;
    b->smem = smem;
    for (auto& a : b->h_insts) a.rpc = rpc;
    cudaError_t e = cudaMemcpy(b->d_insts, b->h_insts.data(), sizeof(sa::SweepArgs) * b->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(e, "copy batch arguments");
    return SA_OK;
}

sa::BatchArgs batch_args(const sa_batch* b, const sa::SweepArgs* insts) {
    sa::BatchArgs a{};
    a.insts = insts;
    a.units = b->d_units;
    a.n_units = (int32_t)b->h_units.size();
    a.counter = b->d_counter;
    a.slot_bytes = (int64_t)b->slot_bytes;
    a.rpc = b->rpc;
    a.tpr = b->tpr;
    a.gstate = b->d_gstate;
    return a;
}

size_t shared_bytes(const sa_batch* b) { return b->smem ? (size_t)b->rpc * b->slot_bytes : 0; }

sa_status capture(sa_batch* b) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    const sa::BatchArgs a = batch_args(b, b->d_insts);
    int le = sa::launch_batch(a, b->is_float, b->kind, b->zbytes, b->rule, b->smem, 0, b->rpc * b->tpr,
                              shared_bytes(b), b->cap, true);
    if (le != 0) return bcuda((cudaError_t)le, "batch kernel attributes");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(e, "begin capture");
    cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), b->cap);
    le = sa::launch_batch(a, b->is_float, b->kind, b->zbytes, b->rule, b->smem, b->blocks, b->rpc * b->tpr,
                          shared_bytes(b), b->cap, false);
    e = cudaStreamEndCapture(b->cap, &g);
    if (le != 0) return bcuda((cudaError_t)le, "batch kernel capture");
    if (e != cudaSuccess) return bcuda(e, "end capture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bcuda(e, "graph instantiate");
    return SA_OK;
}

}  // namespace

extern "C" {

sa_status sa_batch_create(sa_batch** out, const sa_model* const* models, int32_t n_models, const sa_run_params* params) {
    if (!out) return bfail(SA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!models || !params || n_models < 1) return bfail(SA_ERR_INVALID, "empty batch");
    sa_batch* b = new sa_batch();
    cudaGetDevice(&b->device);
    b->n = n_models;
    b->views.resize(n_models);
    for (int i = 0; i < n_models; ++i) {
        if (!models[i] || !sa_internal_model_view(models[i], &b->views[i])) {
            delete b;
            return bfail(SA_ERR_INVALID, "NULL model in batch");
        }
    }
    const sa::ModelView& v0 = b->views[0];
    b->kind = v0.dm.kind;
    b->is_float = v0.is_float;
    b->rule = params[0].rule;
    for (int i = 0; i < n_models; ++i) {
        const sa::ModelView& v = b->views[i];
        const sa_run_params& p = params[i];
        std::string where = " (instance " + std::to_string(i) + ")";
        sa_status st = SA_OK;
        std::string msg;
        if (v.device != b->device) { st = SA_ERR_INVALID; msg = "model on another device"; }
        else if (v.dm.kind != b->kind || v.is_float != b->is_float) { st = SA_ERR_UNSUPPORTED; msg = "a batch needs one model kind and one coefficient class"; }
        else if (p.rule != b->rule) { st = SA_ERR_UNSUPPORTED; msg = "a batch needs one rule"; }
        else if (p.rule < 0 || p.rule > 2) { st = SA_ERR_INVALID; msg = "unknown rule"; }
        else if (p.n_sweeps < 1 || p.n_replicas < 1) { st = SA_ERR_INVALID; msg = "n_sweeps and n_replicas must be positive"; }
        else if (p.rule == SA_OPT_METROPOLIS && v.max_exp > 4) { st = SA_ERR_UNSUPPORTED; msg = "OTM needs exponents <= 4"; }
        else if (p.init_states && !dev_ptr(p.init_states)) { st = SA_ERR_INVALID; msg = "init_states must be device memory"; }
        else if (p.trace) { st = SA_ERR_UNSUPPORTED; msg = "per-attempt traces are not available in batches"; }
        else if (p.best_states || p.best_energies) { st = SA_ERR_UNSUPPORTED; msg = "best-state tracking is not available in batches"; }
        if (st != SA_OK) {
            delete b;
            return bfail(st, msg + where);
        }
        b->zbytes = std::max(b->zbytes, v.zbytes);
    }
    // sizes and offsets
    b->R.resize(n_models);
    b->S.resize(n_models);
    b->st_off.resize(n_models);
    b->en_off.resize(n_models);
    size_t n_states = 0, n_rep = 0, n_tab = 0;
    for (int i = 0; i < n_models; ++i) {
        b->R[i] = params[i].n_replicas;
        b->S[i] = params[i].n_sweeps;
        b->st_off[i] = (int64_t)n_states;
        b->en_off[i] = (int64_t)n_rep;
        n_states += (size_t)b->R[i] * b->views[i].n;
        n_rep += (size_t)b->R[i];
        n_tab += 2 * (size_t)b->S[i];
        b->attempts += (int64_t)b->R[i] * b->S[i] * b->views[i].n;
    }
    // work units: one per replica, by decreasing estimated cost
    for (int i = 0; i < n_models; ++i)
        for (int r = 0; r < b->R[i]; ++r) b->h_units.push_back({i, r});
    std::vector<double> cost(n_models);
    for (int i = 0; i < n_models; ++i) {
        const sa::ModelView& v = b->views[i];
        cost[i] = (double)b->S[i] * ((double)v.n + 64.0 * (double)v.n_levels);
    }
    std::stable_sort(b->h_units.begin(), b->h_units.end(),
                     [&](const sa::BatchUnit& x, const sa::BatchUnit& y) { return cost[x.inst] > cost[y.inst]; });
    // one device allocation: arguments, units, counter, schedules, outputs
    const size_t o_insts = 0;
    const size_t o_units = up256(o_insts + sizeof(sa::SweepArgs) * n_models);
    const size_t o_cnt = up256(o_units + sizeof(sa::BatchUnit) * b->h_units.size());
    const size_t o_tab = up256(o_cnt + 16);
    const size_t o_st = up256(o_tab + sizeof(float) * n_tab);
    const size_t o_en = up256(o_st + sizeof(int32_t) * n_states);
    const size_t o_acc = up256(o_en + 8 * n_rep);
    const size_t total = up256(o_acc + 8 * n_rep);
    cudaError_t e = cudaMalloc(&b->dmem, total);
    if (e != cudaSuccess) {
        delete b;
        return bcuda(e, "cudaMalloc(batch)");
    }
    b->dbytes = total;
    uint8_t* base = static_cast<uint8_t*>(b->dmem);
    b->d_insts = reinterpret_cast<sa::SweepArgs*>(base + o_insts);
    b->d_units = reinterpret_cast<sa::BatchUnit*>(base + o_units);
    b->d_counter = reinterpret_cast<unsigned int*>(base + o_cnt);
    float* d_tab = reinterpret_cast<float*>(base + o_tab);
    b->d_states = reinterpret_cast<int32_t*>(base + o_st);
    b->d_energies = base + o_en;
    b->d_accepts = reinterpret_cast<unsigned long long*>(base + o_acc);
    // schedules
    std::vector<float> tab(n_tab);
    size_t tpos = 0;
    b->h_insts.resize(n_models);
    for (int i = 0; i < n_models; ++i) {
        const sa_run_params& p = params[i];
        const sa::ModelView& v = b->views[i];
        const int32_t S = b->S[i];
        if (const char* err = sa::plan_schedule(v.de_max, v.de_min, S, p.t_max, p.t_min, p.temperatures,
                                                tab.data() + tpos)) {
            cudaFree(b->dmem);
            delete b;
            return bfail(SA_ERR_INVALID, std::string(err) + " (instance " + std::to_string(i) + ")");
        }
        sa::SweepArgs& a = b->h_insts[i];
        a = sa::SweepArgs{};
        a.m = v.dm;
        a.R = b->R[i];
        a.S = S;
        a.key0 = (uint32_t)(p.seed & 0xFFFFFFFFull);
        a.key1 = (uint32_t)(p.seed >> 32);
        a.inst = p.instance_id;
        a.refresh_interval = p.refresh_interval > 0 ? p.refresh_interval : 50;
        a.speculate = (p.flags & SA_FLAG_NO_SPECULATION) ? 0 : 1;
        a.beta = d_tab + tpos;
        a.ratio = d_tab + tpos + S;
        a.init_states = p.init_states;
        a.out_states = b->d_states + b->st_off[i];
        a.out_energies = reinterpret_cast<uint8_t*>(b->d_energies) + 8 * b->en_off[i];
        a.out_accepts = b->d_accepts + b->en_off[i];
        a.trace = nullptr;
        a.trace_R = 0;
        a.energy_trace = p.energy_trace;
        a.drift_bits = nullptr;
        a.gstate = nullptr;
        tpos += 2 * (size_t)S;
    }
    e = cudaMemcpy(d_tab, tab.data(), sizeof(float) * n_tab, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_units, b->h_units.data(), sizeof(sa::BatchUnit) * b->h_units.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(b->dmem);
        delete b;
        return bcuda(e, "copy batch tables");
    }
    // heuristic shape: threads per replica from the cost-weighted mean level width
    double wsum = 0, csum = 0;
    for (int i = 0; i < n_models; ++i) {
        const sa::ModelView& v = b->views[i];
        const double c = cost[i] * b->R[i];
        wsum += c * (double)v.n / (double)std::max(1, v.n_levels);
        csum += c;
    }
    const double mean_w = wsum / std::max(1.0, csum);
    int tpr = std::min(256, std::max(32, ((int)std::ceil(mean_w / 2.0) + 31) / 32 * 32));
    sa_status st = apply_shape(b, tpr, 0);
    if (st == SA_OK) {
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = bcuda(e, "create stream");
    }
    if (st == SA_OK) st = capture(b);
    if (st != SA_OK) {
        sa_batch_destroy(b);
        return st;
    }
    *out = b;
    return SA_OK;
}

sa_status sa_batch_run(sa_batch* b, void* stream) {
    if (!b || !b->exec) return bfail(SA_ERR_INVALID, "NULL batch");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return bcuda(e, "graph launch");
    return SA_OK;
}

sa_status sa_batch_autotune(sa_batch* b, int32_t trial_sweeps, void* stream) {
    if (!b) return bfail(SA_ERR_INVALID, "NULL batch");
    if (trial_sweeps < 1) trial_sweeps = 1;
    cudaStream_t st = (cudaStream_t)stream;
    const int cands[] = {32, 64, 96, 128, 256};
    int best_tpr = b->tpr, best_rpc = b->rpc;
    float best = INFINITY;
    sa::SweepArgs* d_trial = nullptr;
    cudaError_t e = cudaMalloc(&d_trial, sizeof(sa::SweepArgs) * b->n);
    if (e != cudaSuccess) return bcuda(e, "cudaMalloc(trial)");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int tpr : cands) {
        if (apply_shape(b, tpr, 0) != SA_OK) continue;
        std::vector<sa::SweepArgs> trial = b->h_insts;
        for (auto& a : trial) a.S = std::min(a.S, trial_sweeps);
        cudaMemcpy(d_trial, trial.data(), sizeof(sa::SweepArgs) * b->n, cudaMemcpyHostToDevice);
        const sa::BatchArgs a = batch_args(b, d_trial);
        float ms_best = INFINITY;
        for (int rep = 0; rep < 2; ++rep) {
            cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned int), st);
            cudaEventRecord(e0, st);
            int le = sa::launch_batch(a, b->is_float, b->kind, b->zbytes, b->rule, b->smem, b->blocks,
                                      b->rpc * b->tpr, shared_bytes(b), st, true);
            cudaEventRecord(e1, st);
            if (le != 0) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_best = std::min(ms_best, ms);
        }
        if (ms_best < best) {
            best = ms_best;
            best_tpr = b->tpr;
            best_rpc = b->rpc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_trial);
    cudaGetLastError();
    sa_status s2 = apply_shape(b, best_tpr, best_rpc);
    if (s2 != SA_OK) return s2;
    b->last_ms = best;
    return capture(b);
}

sa_status sa_batch_result(const sa_batch* b, int32_t i, int32_t* states, void* energies, uint64_t* accepts,
                          void* stream) {
    if (!b || i < 0 || i >= b->n) return bfail(SA_ERR_INVALID, "bad batch or instance index");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ns = (size_t)b->R[i] * b->views[i].n, nr = (size_t)b->R[i];
    cudaError_t e = cudaSuccess;
    if (states) e = cudaMemcpyAsync(states, b->d_states + b->st_off[i], 4 * ns, cudaMemcpyDefault, st);
    if (e == cudaSuccess && energies)
        e = cudaMemcpyAsync(energies, reinterpret_cast<const uint8_t*>(b->d_energies) + 8 * b->en_off[i], 8 * nr,
                            cudaMemcpyDefault, st);
    if (e == cudaSuccess && accepts) e = cudaMemcpyAsync(accepts, b->d_accepts + b->en_off[i], 8 * nr, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bcuda(e, "batch result");
    return SA_OK;
}

sa_status sa_batch_get_info(const sa_batch* b, sa_batch_info* info) {
    if (!b || !info) return bfail(SA_ERR_INVALID, "NULL argument");
    info->n_instances = b->n;
    info->n_units = (int32_t)b->h_units.size();
    info->replicas_per_block = b->rpc;
    info->threads_per_replica = b->tpr;
    info->blocks = b->blocks;
    info->state_in_global = b->smem ? 0 : 1;
    info->attempts = b->attempts;
    info->device_bytes = (int64_t)(b->dbytes + b->gstate_bytes);
    info->autotune_ms = b->last_ms;
    return SA_OK;
}

void sa_batch_destroy(sa_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_gstate) cudaFree(b->d_gstate);
    if (b->dmem) cudaFree(b->dmem);
    delete b;
}

}  // extern "C"
