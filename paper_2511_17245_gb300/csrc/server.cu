// server.cu -- a request server for SA solves with continuous batching.
//
// Requests (model + sa_run_params) enter a FIFO queue.  A dispatcher thread
// admits them in order, skipping ahead past a request that does not fit yet
// (backfill), whenever a request slot is free and the request's device bytes
// (model, outputs, schedule, replica state that does not fit a shared-memory
// region) fit the budget.  Admission turns the request's R replicas into R
// units of one work queue: the request's run arguments go into a host-mapped
// table, its units into a host-mapped ring, and the published tail moves on.
// One persistent kernel (serve_kernel.cu) drains the queue: each of its thread
// groups claims the next unit, runs that replica and, when the last unit of a
// request finishes, raises the request's done flag in host memory.  Requests
// admitted while others run therefore share the GPU replica by replica, and a
// finished request's memory and slot are released at once.  The kernel leaves
// when no admitted request is left (the dispatcher raises a stop word; its
// groups also leave after a long, bounded idle period); the dispatcher launches
// it again whenever admitted work is waiting and no kernel runs.  Every wait in
// this file is bounded, and the dispatcher makes no call that synchronises the
// device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "sa.h"
#include "sa_internal.h"

extern "C" int sa_internal_model_view(const sa_model* M, sa::ModelView* v);
extern "C" void sa_internal_set_error(const char* msg);
extern "C" __attribute__((visibility("hidden"))) int64_t sa_internal_model_bytes(const sa_model* M);

namespace {

using Clock = std::chrono::steady_clock;

constexpr uint32_t kRingCap = 1u << 20;      // units in flight (published, not finished)
constexpr int kMaxRunning = 8192;
// Polls of an empty queue (about 2 us each) before a group leaves on its own.
// Groups normally leave when the dispatcher raises the stop word (no admitted
// request left); this bound only ends a kernel whose server stopped answering.
constexpr uint32_t kIdlePolls = 100000000u;

sa_status sfail(sa_status st, const std::string& msg) {
    sa_internal_set_error(msg.c_str());
    return st;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Request {
    uint64_t ticket = 0;
    const sa_model* model = nullptr;
    sa_run_params params{};
    std::vector<double> temps;   // copy of params.temperatures
    sa::ModelView view{};
    int32_t n = 0;
    bool is_float = false;
    int zbytes = 2;              // state offsets in the serving kernel
    int64_t rep_bytes = 0;
    bool slab = false;           // replica state in global memory
    int64_t bytes = 0;           // device bytes charged against the budget
    int state = SA_REQ_QUEUED;
    sa_status status = SA_OK;
    std::string error;
    int slot = -1;
    void* dmem = nullptr;        // outputs, schedule and state slab
    size_t o_en = 0, o_acc = 0, o_tab = 0, o_slab = 0;
    std::vector<int32_t> h_states;
    std::vector<uint8_t> h_en;
    std::vector<uint64_t> h_acc;
    Clock::time_point t_submit, t_start, t_end;
};

}  // namespace

struct sa_server {
    sa_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Request*> reqs;
    int64_t in_use = 0, peak = 0;
    uint64_t next_ticket = 1;
    int64_t completed = 0, failed = 0, cancelled = 0;
    int64_t attempts_done = 0, units_done = 0, launches = 0;
    std::vector<double> latencies_ms;
    Clock::time_point t_first_submit{}, t_last_done{};
    bool any_submit = false;
    std::atomic<bool> stop{false};
    std::thread worker;

    // serving engine
    cudaStream_t kstream = nullptr, cstream = nullptr;
    cudaEvent_t kdone = nullptr;
    bool launched = false;
    sa::ServeReq* h_reqs = nullptr;     // host-mapped tables (device aliases below)
    sa::ServeUnit* h_units = nullptr;
    sa::ServeCtl* h_ctl = nullptr;
    unsigned int* h_done = nullptr;
    sa::ServeArgs args{};
    uint32_t published = 0;
    int64_t units_finished = 0;
    std::vector<int> free_slots;
    std::vector<Request*> slot_req;
    int grid = 0;
    size_t shared = 0;
};

namespace {

bool kernel_running(sa_server* s) { return s->launched && cudaEventQuery(s->kdone) == cudaErrorNotReady; }

// Plans a request for the serving kernel: state width, layout and placement.
void plan_request(const sa_server* s, Request* r) {
    const sa::ModelView& v = r->view;
    uint32_t maxw = v.dm.max_width;
    r->zbytes = maxw <= 0xFFFFu ? 2 : 4;
    sa::RunPlan pl{};
    r->rep_bytes = sa::plan_layout(sa::plan_model(v), r->zbytes, s->args.tpr, &pl);
    r->slab = r->rep_bytes > s->args.slot_bytes;
    const int64_t R = r->params.n_replicas, S = r->params.n_sweeps, n = v.n;
    int64_t b = (int64_t)round_up((size_t)(R * n * 4), 256) + 2 * (int64_t)round_up((size_t)(R * 8), 256) +
                (int64_t)round_up((size_t)(S * 8), 256);
    if (r->slab) b += R * r->rep_bytes;
    r->bytes = b;
}

// Admits request r into slot `slot`: device memory, schedule, run arguments,
// units.  Called with the lock held.  Returns false (request failed) on error.
bool admit(sa_server* s, Request* r, int slot) {
    const sa::ModelView& v = r->view;
    const int32_t R = r->params.n_replicas, S = r->params.n_sweeps, n = v.n;
    std::vector<float> tab(2 * (size_t)S);
    const sa_run_params& p = r->params;
    if (const char* err = sa::plan_schedule(v.de_max, v.de_min, S, p.t_max, p.t_min,
                                            r->temps.empty() ? nullptr : r->temps.data(), tab.data())) {
        r->status = SA_ERR_INVALID;
        r->error = err;
        return false;
    }
    const size_t o_st = 0;
    r->o_en = round_up(o_st + (size_t)R * n * 4, 256);
    r->o_acc = round_up(r->o_en + (size_t)R * 8, 256);
    r->o_tab = round_up(r->o_acc + (size_t)R * 8, 256);
    r->o_slab = round_up(r->o_tab + tab.size() * 4, 256);
    const size_t total = r->o_slab + (r->slab ? (size_t)R * (size_t)r->rep_bytes : 0);
    cudaError_t e = cudaMallocAsync(&r->dmem, total, s->cstream);
    uint8_t* d = static_cast<uint8_t*>(r->dmem);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d + r->o_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, s->cstream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->args.req_units_done + slot, 0, 4, s->cstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cstream);
    if (e != cudaSuccess) {
        r->status = e == cudaErrorMemoryAllocation ? SA_ERR_OOM : SA_ERR_CUDA;
        r->error = std::string("request setup: ") + cudaGetErrorString(e);
        if (r->dmem) cudaFreeAsync(r->dmem, s->cstream);
        r->dmem = nullptr;
        return false;
    }
    sa::SweepArgs a{};
    a.m = v.dm;
    a.R = R;
    a.S = S;
    a.key0 = (uint32_t)(p.seed & 0xFFFFFFFFull);
    a.key1 = (uint32_t)(p.seed >> 32);
    a.inst = p.instance_id;
    a.refresh_interval = p.refresh_interval > 0 ? p.refresh_interval : 50;
    a.speculate = (p.flags & SA_FLAG_NO_SPECULATION) ? 0 : 1;
    a.beta = reinterpret_cast<const float*>(d + r->o_tab);
    a.ratio = a.beta + S;
    a.out_states = reinterpret_cast<int32_t*>(d + o_st);
    a.out_energies = d + r->o_en;
    a.out_accepts = reinterpret_cast<unsigned long long*>(d + r->o_acc);
    a.gstate = r->slab ? d + r->o_slab : nullptr;
    sa::RunPlan pl{};
    sa::plan_layout(sa::plan_model(v), r->zbytes, s->args.tpr, &pl);
    pl.rpc = s->args.rpc;
    sa::plan_apply(pl, a);
    sa::ServeReq& q = s->h_reqs[slot];
    q.args = a;
    q.variant = sa::serve_variant(p.rule, v.dm.kind, v.is_float, r->zbytes);
    q.n_units = R;
    s->h_done[slot] = 0u;
    for (int32_t i = 0; i < R; ++i) s->h_units[(s->published + (uint32_t)i) & (kRingCap - 1u)] = sa::ServeUnit{slot, i};
    std::atomic_thread_fence(std::memory_order_seq_cst);   // table and units before the tail
    s->published += (uint32_t)R;
    s->h_ctl->tail = s->published;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    r->slot = slot;
    s->slot_req[slot] = r;
    r->t_start = Clock::now();
    r->state = SA_REQ_RUNNING;
    return true;
}

void release(sa_server* s, Request* r) {
    if (r->dmem) cudaFreeAsync(r->dmem, s->cstream);
    r->dmem = nullptr;
    if (r->slot >= 0) {
        s->slot_req[r->slot] = nullptr;
        s->free_slots.push_back(r->slot);
        r->slot = -1;
    }
    s->in_use -= r->bytes;
}

// A request whose done flag is up: copy its results to the host, release it.
void finish(sa_server* s, Request* r) {
    const size_t R = r->params.n_replicas, n = r->n;
    const uint8_t* d = static_cast<const uint8_t*>(r->dmem);
    r->h_states.resize(R * n);
    r->h_en.resize(R * 8);
    r->h_acc.resize(R);
    cudaError_t e = cudaMemcpyAsync(r->h_states.data(), d, R * n * 4, cudaMemcpyDeviceToHost, s->cstream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->h_en.data(), d + r->o_en, R * 8, cudaMemcpyDeviceToHost, s->cstream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r->h_acc.data(), d + r->o_acc, R * 8, cudaMemcpyDeviceToHost, s->cstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cstream);
    r->t_end = Clock::now();
    s->units_finished += (int64_t)R;
    s->units_done += (int64_t)R;
    if (e == cudaSuccess) {
        r->state = SA_REQ_DONE;
        s->completed++;
        s->attempts_done += (int64_t)r->params.n_replicas * r->params.n_sweeps * r->n;
        s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_end - r->t_submit).count());
        s->t_last_done = r->t_end;
    } else {
        r->state = SA_REQ_FAILED;
        r->status = SA_ERR_CUDA;
        r->error = std::string("result copy: ") + cudaGetErrorString(e);
        s->failed++;
    }
    release(s, r);
}

void fail_running(sa_server* s, const std::string& why) {
    for (size_t i = 0; i < s->slot_req.size(); ++i) {
        Request* r = s->slot_req[i];
        if (!r) continue;
        r->state = SA_REQ_FAILED;
        r->status = SA_ERR_CUDA;
        r->error = why;
        r->t_end = Clock::now();
        s->failed++;
        s->units_finished += r->params.n_replicas;
        release(s, r);
    }
}

bool launch_kernel(sa_server* s) {
    s->h_ctl->stop = 0u;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    int le = sa::launch_serve(s->args, s->grid, s->shared, s->kstream);
    if (le != 0) return false;
    cudaEventRecord(s->kdone, s->kstream);
    s->launched = true;
    s->launches++;
    return true;
}

void dispatcher(sa_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop.load()) {
        bool progressed = false;
        // completions: done flags raised by the kernel in host memory
        int active = 0;
        for (size_t i = 0; i < s->slot_req.size(); ++i) {
            Request* r = s->slot_req[i];
            if (!r) continue;
            if (reinterpret_cast<volatile unsigned int*>(s->h_done)[i] != 0u) {
                std::atomic_thread_fence(std::memory_order_acquire);
                finish(s, r);
                progressed = true;
            } else {
                ++active;
            }
        }
        if (progressed) s->cv_done.notify_all();
        // admissions: FIFO with backfill
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            Request* r = s->reqs[*it];
            if (r->state != SA_REQ_QUEUED) {
                it = s->queue.erase(it);
                continue;
            }
            if (s->free_slots.empty()) break;
            const int64_t inflight = (int64_t)s->published - s->units_finished;
            if (s->in_use + r->bytes > (int64_t)s->cfg.budget_bytes ||
                inflight + r->params.n_replicas > (int64_t)kRingCap) {
                ++it;
                continue;
            }
            const int slot = s->free_slots.back();
            s->free_slots.pop_back();
            s->in_use += r->bytes;
            s->peak = std::max(s->peak, s->in_use);
            if (!admit(s, r, slot)) {
                s->free_slots.push_back(slot);
                s->in_use -= r->bytes;
                r->state = SA_REQ_FAILED;
                r->t_end = Clock::now();
                s->failed++;
                s->cv_done.notify_all();
            } else {
                ++active;
            }
            it = s->queue.erase(it);
            progressed = true;
        }
        // the persistent kernel: running while admitted work waits
        if (s->launched && !kernel_running(s)) {
            const cudaError_t ke = cudaEventQuery(s->kdone);
            if (ke != cudaSuccess && ke != cudaErrorNotReady) {
                fail_running(s, std::string("serving kernel: ") + cudaGetErrorString(ke));
                s->cv_done.notify_all();
                active = 0;
            }
        }
        if (active > 0) {
            if (s->h_ctl->stop != 0u) s->h_ctl->stop = 0u;
            if (!kernel_running(s) && !launch_kernel(s)) {
                fail_running(s, "serving kernel launch failed");
                s->cv_done.notify_all();
            }
        } else if (kernel_running(s)) {
            s->h_ctl->stop = 1u;   // nothing admitted: let the groups leave
        }
        if (!progressed) s->cv_work.wait_for(lk, std::chrono::microseconds(active > 0 ? 50 : 2000));
    }
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = p * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

void free_engine(sa_server* s) {
    if (s->kstream) cudaStreamDestroy(s->kstream);
    if (s->cstream) cudaStreamDestroy(s->cstream);
    if (s->kdone) cudaEventDestroy(s->kdone);
    if (s->args.head) cudaFree(s->args.head);
    if (s->h_reqs) cudaFreeHost(s->h_reqs);
    if (s->h_units) cudaFreeHost(s->h_units);
    if (s->h_ctl) cudaFreeHost(s->h_ctl);
    if (s->h_done) cudaFreeHost(s->h_done);
}

}  // namespace

extern "C" {

sa_status sa_server_create(sa_server** out, const sa_server_config* cfg) {
    if (!out || !cfg) return sfail(SA_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (cfg->budget_bytes == 0 || cfg->max_running < 1 || cfg->max_running > kMaxRunning)
        return sfail(SA_ERR_INVALID, "budget must be positive and max_running in 1..8192");
    const int tpr = cfg->threads_per_replica > 0 ? cfg->threads_per_replica : 256;
    if (tpr != 64 && tpr != 128 && tpr != 256) return sfail(SA_ERR_INVALID, "threads_per_replica must be 0, 64, 128 or 256");
    sa_server* s = new sa_server();
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    const int nreq = cfg->max_running;
    cudaError_t e = cudaStreamCreateWithFlags(&s->kstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->kdone, cudaEventDisableTiming);
    const unsigned int fl = cudaHostAllocMapped | cudaHostAllocPortable;
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_reqs, sizeof(sa::ServeReq) * nreq, fl);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_units, sizeof(sa::ServeUnit) * kRingCap, fl);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_ctl, sizeof(sa::ServeCtl), fl);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&s->h_done, sizeof(unsigned int) * nreq, fl);
    unsigned int* dmem = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void**)&dmem, sizeof(unsigned int) * (nreq + 4));
    if (e == cudaSuccess) e = cudaMemset(dmem, 0, sizeof(unsigned int) * (nreq + 4));
    if (e != cudaSuccess) {
        free_engine(s);
        delete s;
        return sfail(e == cudaErrorMemoryAllocation ? SA_ERR_OOM : SA_ERR_CUDA,
                     std::string("server create: ") + cudaGetErrorString(e));
    }
    std::memset(s->h_reqs, 0, sizeof(sa::ServeReq) * nreq);
    std::memset(s->h_done, 0, sizeof(unsigned int) * nreq);
    s->h_ctl->tail = 0u;
    s->h_ctl->stop = 0u;
    sa::ServeArgs& a = s->args;
    void* dp = nullptr;
    cudaHostGetDevicePointer(&dp, s->h_reqs, 0);
    a.reqs = static_cast<const sa::ServeReq*>(dp);
    cudaHostGetDevicePointer(&dp, s->h_units, 0);
    a.units = static_cast<const sa::ServeUnit*>(dp);
    cudaHostGetDevicePointer(&dp, s->h_ctl, 0);
    a.ctl = static_cast<const sa::ServeCtl*>(dp);
    cudaHostGetDevicePointer(&dp, s->h_done, 0);
    a.req_done = static_cast<unsigned int*>(dp);
    a.head = dmem;
    a.req_units_done = dmem + 4;
    a.cap = kRingCap;
    a.tpr = tpr;
    a.rpc = 512 / tpr;
    a.idle_polls = kIdlePolls;
    const size_t avail = (size_t)sa::sweep_max_shared_optin() - sa::serve_static_shared();
    a.slot_bytes = (int64_t)(avail / (size_t)a.rpc / 16 * 16);
    s->shared = (size_t)a.slot_bytes * (size_t)a.rpc;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    s->grid = sms;   // one block of 512 threads per SM (the state regions fill its shared memory)
    int le = sa::launch_serve(a, 0, s->shared, s->kstream);
    if (le != 0) {
        free_engine(s);
        delete s;
        return sfail(SA_ERR_CUDA, std::string("serving kernel attributes: ") + cudaGetErrorString((cudaError_t)le));
    }
    s->slot_req.assign(nreq, nullptr);
    for (int i = nreq - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->worker = std::thread(dispatcher, s);
    *out = s;
    return SA_OK;
}

sa_status sa_server_submit(sa_server* s, const sa_model* model, const sa_run_params* params, uint64_t* ticket) {
    if (!s || !model || !params || !ticket) return sfail(SA_ERR_INVALID, "NULL argument");
    sa::ModelView v;
    if (!sa_internal_model_view(model, &v)) return sfail(SA_ERR_INVALID, "bad model");
    int dev = 0;
    cudaGetDevice(&dev);
    if (v.device != s->device) return sfail(SA_ERR_INVALID, "model belongs to another device than the server");
    if (params->n_sweeps < 1 || params->n_replicas < 1 || params->rule < 0 || params->rule > 2)
        return sfail(SA_ERR_INVALID, "bad run parameters");
    if (params->trace || params->energy_trace || params->report || params->init_states || params->best_states ||
        params->best_energies)
        return sfail(SA_ERR_UNSUPPORTED, "served requests take no traces, report, initial or best states");
    if (params->rule == SA_OPT_METROPOLIS && v.max_exp > 4)
        return sfail(SA_ERR_UNSUPPORTED, "OTM needs exponents <= 4");
    if (params->n_replicas > (int32_t)kRingCap) return sfail(SA_ERR_UNSUPPORTED, "too many replicas for the work queue");
    Request* r = new Request();
    r->model = model;
    r->params = *params;
    if (params->temperatures) {
        r->temps.assign(params->temperatures, params->temperatures + params->n_sweeps);
        r->params.temperatures = nullptr;
    }
    r->view = v;
    r->n = v.n;
    r->is_float = v.is_float != 0;
    plan_request(s, r);
    r->bytes += sa_internal_model_bytes(model);
    if (r->bytes > (int64_t)s->cfg.budget_bytes) {
        delete r;
        return sfail(SA_ERR_OOM, "request needs more device memory than the whole budget");
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->queue.push_back(r->ticket);
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first_submit = r->t_submit;
        }
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return SA_OK;
}

sa_status sa_server_poll(sa_server* s, uint64_t ticket, int32_t* state) {
    if (!s || !state) return sfail(SA_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(SA_ERR_INVALID, "unknown ticket");
    *state = it->second->state;
    return SA_OK;
}

sa_status sa_server_wait(sa_server* s, uint64_t ticket, int64_t timeout_us) {
    if (!s) return sfail(SA_ERR_INVALID, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(SA_ERR_INVALID, "unknown ticket");
    Request* r = it->second;
    const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    while (r->state == SA_REQ_QUEUED || r->state == SA_REQ_RUNNING) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            (r->state == SA_REQ_QUEUED || r->state == SA_REQ_RUNNING))
            return sfail(SA_ERR_TIMEOUT, "request not finished within the timeout");
    }
    return r->state == SA_REQ_DONE ? SA_OK : sfail(r->state == SA_REQ_CANCELLED ? SA_ERR_INVALID : r->status,
                                                    r->state == SA_REQ_CANCELLED ? "request cancelled" : r->error);
}

sa_status sa_server_cancel(sa_server* s, uint64_t ticket) {
    if (!s) return sfail(SA_ERR_INVALID, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(SA_ERR_INVALID, "unknown ticket");
    if (it->second->state != SA_REQ_QUEUED) return sfail(SA_ERR_BUSY, "only queued requests can be cancelled");
    it->second->state = SA_REQ_CANCELLED;
    s->cancelled++;
    s->cv_done.notify_all();
    return SA_OK;
}

sa_status sa_server_result(sa_server* s, uint64_t ticket, int32_t* states, void* energies, uint64_t* accepts,
                           double* latency_ms) {
    if (!s) return sfail(SA_ERR_INVALID, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(SA_ERR_INVALID, "unknown ticket");
    Request* r = it->second;
    if (r->state != SA_REQ_DONE) return sfail(SA_ERR_BUSY, "request not done");
    const size_t R = r->params.n_replicas, n = r->n;
    if (states) std::memcpy(states, r->h_states.data(), R * n * 4);
    if (energies) std::memcpy(energies, r->h_en.data(), R * 8);
    if (accepts) std::memcpy(accepts, r->h_acc.data(), R * 8);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_end - r->t_submit).count();
    s->reqs.erase(it);
    delete r;
    return SA_OK;
}

sa_status sa_server_get_stats(sa_server* s, sa_server_stats* st) {
    if (!s || !st) return sfail(SA_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(st, 0, sizeof(*st));
    st->completed = s->completed;
    st->failed = s->failed;
    st->cancelled = s->cancelled;
    int64_t q = 0, run = 0;
    for (auto& kv : s->reqs) {
        if (kv.second->state == SA_REQ_QUEUED) ++q;
        if (kv.second->state == SA_REQ_RUNNING) ++run;
    }
    st->queued = q;
    st->running = run;
    st->device_bytes_in_use = s->in_use;
    st->device_bytes_peak = s->peak;
    st->attempts = s->attempts_done;
    st->p50_latency_ms = percentile(s->latencies_ms, 0.50);
    st->p99_latency_ms = percentile(s->latencies_ms, 0.99);
    const double span = s->any_submit && s->completed > 0
                            ? std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count()
                            : 0.0;
    st->attempts_per_s = span > 0 ? (double)s->attempts_done / span : 0.0;
    st->units_done = s->units_done;
    st->kernel_launches = s->launches;
    return SA_OK;
}

void sa_server_destroy(sa_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& kv : s->reqs)
            if (kv.second->state == SA_REQ_QUEUED) kv.second->state = SA_REQ_CANCELLED;
    }
    // let running requests finish (bounded), then stop the dispatcher and the kernel
    const auto deadline = Clock::now() + std::chrono::seconds(600);
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            bool running = false;
            for (auto& kv : s->reqs)
                if (kv.second->state == SA_REQ_RUNNING) running = true;
            if (!running || Clock::now() > deadline) break;
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    s->stop.store(true);
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->h_ctl) s->h_ctl->stop = 1u;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    // the groups leave once the queue is empty; wait for the kernel (bounded)
    const auto kdeadline = Clock::now() + std::chrono::seconds(600);
    while (s->launched && cudaEventQuery(s->kdone) == cudaErrorNotReady && Clock::now() < kdeadline)
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    for (auto& kv : s->reqs) {
        Request* r = kv.second;
        if (r->dmem) cudaFreeAsync(r->dmem, s->cstream);
        delete r;
    }
    cudaStreamSynchronize(s->cstream);
    free_engine(s);
    delete s;
}

}  // extern "C"
