// server.cu -- a request loop for SA solves with continuous admission.
//
// Requests (model + sa_run_params) enter a FIFO queue.  A dispatcher thread
// admits queued requests in order, skipping ahead past a request that does not
// fit yet (backfill), whenever a stream of the pool is free and the request's
// device bytes fit the budget.  An admitted request gets its own stream: the
// server allocates its output buffers there (stream-ordered), enqueues sa_run
// with device outputs (asynchronous), the copies of the results into pinned
// host memory and an event.  Requests admitted while others run execute
// concurrently on the device.  Completed requests release their device memory
// and stream at once, so waiting requests enter as soon as room appears.
// Every wait in this file is bounded.
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

sa_status sfail(sa_status st, const std::string& msg) {
    sa_internal_set_error(msg.c_str());
    return st;
}

struct Request {
    uint64_t ticket = 0;
    const sa_model* model = nullptr;
    sa_run_params params{};
    std::vector<double> temps;   // copy of params.temperatures
    int32_t n = 0;
    bool is_float = false;
    int64_t bytes = 0;           // device bytes charged against the budget
    int state = SA_REQ_QUEUED;
    sa_status status = SA_OK;
    std::string error;
    int stream_slot = -1;
    int32_t* d_states = nullptr;
    void* d_en = nullptr;
    unsigned long long* d_acc = nullptr;
    int32_t* h_states = nullptr;  // pinned
    void* h_en = nullptr;
    unsigned long long* h_acc = nullptr;
    cudaEvent_t done_ev = nullptr;
    Clock::time_point t_submit, t_start, t_end;
};

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct sa_server {
    sa_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Request*> reqs;
    std::vector<cudaStream_t> streams;
    std::vector<int> stream_busy;
    int64_t in_use = 0, peak = 0;
    uint64_t next_ticket = 1;
    int64_t completed = 0, failed = 0, cancelled = 0;
    int64_t attempts_done = 0;
    std::vector<double> latencies_ms;
    Clock::time_point t_first_submit{}, t_last_done{};
    bool any_submit = false;
    std::atomic<bool> stop{false};
    std::thread worker;
};

namespace {

int64_t request_bytes(const Request& r, const sa::ModelView& v) {
    const int64_t R = r.params.n_replicas, S = r.params.n_sweeps, n = v.n;
    int64_t b = 0;
    b += round_up((size_t)(R * n * 4), 256) + round_up((size_t)(R * 8), 256) * 2;   // outputs
    b += round_up((size_t)(S * 8), 256);                                            // schedule
    // replica state slab if it cannot stay on chip (upper bound)
    const int64_t fsize = v.is_float ? 4 : 8;
    const int64_t rep = (int64_t)round_up((size_t)(n * v.zbytes), 16) + v.cache_elems * fsize + 4096;
    if (rep > 200 * 1024 || (r.params.flags & SA_FLAG_STATE_IN_GLOBAL)) b += R * rep;
    return b;
}

void free_request_device(Request* r, cudaStream_t st) {
    if (r->d_states) cudaFreeAsync(r->d_states, st);
    if (r->d_en) cudaFreeAsync(r->d_en, st);
    if (r->d_acc) cudaFreeAsync(r->d_acc, st);
    r->d_states = nullptr;
    r->d_en = nullptr;
    r->d_acc = nullptr;
    if (r->done_ev) cudaEventDestroy(r->done_ev);
    r->done_ev = nullptr;
}

// Starts a request on stream slot `slot`.  Called with the lock held.
void start_request(sa_server* s, Request* r, int slot) {
    cudaStream_t st = s->streams[slot];
    const size_t R = r->params.n_replicas, n = r->n;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
        return e == cudaSuccess;
    };
    ok(cudaMallocAsync((void**)&r->d_states, R * n * 4, st));
    ok(cudaMallocAsync(&r->d_en, R * 8, st));
    ok(cudaMallocAsync((void**)&r->d_acc, R * 8, st));
    ok(cudaMallocHost((void**)&r->h_states, R * n * 4));
    ok(cudaMallocHost(&r->h_en, R * 8));
    ok(cudaMallocHost((void**)&r->h_acc, R * 8));
    ok(cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming));
    r->stream_slot = slot;
    r->t_start = Clock::now();
    if (e != cudaSuccess) {
        r->status = e == cudaErrorMemoryAllocation ? SA_ERR_OOM : SA_ERR_CUDA;
        r->error = std::string("request setup: ") + cudaGetErrorString(e);
        r->state = SA_REQ_FAILED;
        return;
    }
    sa_run_params p = r->params;
    p.temperatures = r->temps.empty() ? nullptr : r->temps.data();
    p.report = nullptr;
    sa_status rc = sa_run(r->model, &p, r->d_states, r->d_en, (uint64_t*)r->d_acc, st);
    if (rc != SA_OK) {
        r->status = rc;
        r->error = sa_last_error();
        r->state = SA_REQ_FAILED;
        return;
    }
    ok(cudaMemcpyAsync(r->h_states, r->d_states, R * n * 4, cudaMemcpyDeviceToHost, st));
    ok(cudaMemcpyAsync(r->h_en, r->d_en, R * 8, cudaMemcpyDeviceToHost, st));
    ok(cudaMemcpyAsync(r->h_acc, r->d_acc, R * 8, cudaMemcpyDeviceToHost, st));
    ok(cudaEventRecord(r->done_ev, st));
    if (e != cudaSuccess) {
        r->status = SA_ERR_CUDA;
        r->error = std::string("request enqueue: ") + cudaGetErrorString(e);
        r->state = SA_REQ_FAILED;
        return;
    }
    r->state = SA_REQ_RUNNING;
}

void finish(sa_server* s, Request* r) {
    r->t_end = Clock::now();
    if (r->state == SA_REQ_RUNNING) {
        r->state = SA_REQ_DONE;
        s->completed++;
        s->attempts_done += (int64_t)r->params.n_replicas * r->params.n_sweeps * r->n;
        s->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_end - r->t_submit).count());
        s->t_last_done = r->t_end;
    } else {
        s->failed++;
    }
    free_request_device(r, r->stream_slot >= 0 ? s->streams[r->stream_slot] : (cudaStream_t)0);
    if (r->stream_slot >= 0) s->stream_busy[r->stream_slot] = 0;
    r->stream_slot = -1;
    s->in_use -= r->bytes;
}

void dispatcher(sa_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop.load()) {
        bool progressed = false;
        // completions
        for (auto& kv : s->reqs) {
            Request* r = kv.second;
            if (r->state == SA_REQ_RUNNING) {
                const cudaError_t q = cudaEventQuery(r->done_ev);
                if (q == cudaSuccess) {
                    finish(s, r);
                    progressed = true;
                } else if (q != cudaErrorNotReady) {
                    r->status = SA_ERR_CUDA;
                    r->error = std::string("request: ") + cudaGetErrorString(q);
                    r->state = SA_REQ_FAILED;
                    finish(s, r);
                    progressed = true;
                }
            } else if (r->state == SA_REQ_FAILED && r->stream_slot >= 0) {
                finish(s, r);
                progressed = true;
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
            int slot = -1;
            for (size_t i = 0; i < s->streams.size(); ++i)
                if (!s->stream_busy[i]) { slot = (int)i; break; }
            if (slot < 0) break;
            if (s->in_use + r->bytes > (int64_t)s->cfg.budget_bytes) { ++it; continue; }
            s->stream_busy[slot] = 1;
            s->in_use += r->bytes;
            s->peak = std::max(s->peak, s->in_use);
            start_request(s, r, slot);
            if (r->state == SA_REQ_FAILED) finish(s, r);
            it = s->queue.erase(it);
            progressed = true;
        }
        bool running = false;
        for (auto& kv : s->reqs)
            if (kv.second->state == SA_REQ_RUNNING) { running = true; break; }
        if (!progressed) {
            if (running) s->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
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

}  // namespace

extern "C" {

sa_status sa_server_create(sa_server** out, const sa_server_config* cfg) {
    if (!out || !cfg) return sfail(SA_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (cfg->budget_bytes == 0 || cfg->n_streams < 1 || cfg->n_streams > 1024)
        return sfail(SA_ERR_INVALID, "budget must be positive and n_streams in 1..1024");
    sa_server* s = new sa_server();
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    s->streams.resize(cfg->n_streams);
    s->stream_busy.assign(cfg->n_streams, 0);
    for (auto& st : s->streams) {
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (auto& x : s->streams)
                if (x) cudaStreamDestroy(x);
            delete s;
            return sfail(SA_ERR_CUDA, std::string("stream create: ") + cudaGetErrorString(e));
        }
    }
    s->worker = std::thread(dispatcher, s);
    *out = s;
    return SA_OK;
}

sa_status sa_server_submit(sa_server* s, const sa_model* model, const sa_run_params* params, uint64_t* ticket) {
    if (!s || !model || !params || !ticket) return sfail(SA_ERR_INVALID, "NULL argument");
    sa::ModelView v;
    if (!sa_internal_model_view(model, &v)) return sfail(SA_ERR_INVALID, "bad model");
    if (params->n_sweeps < 1 || params->n_replicas < 1 || params->rule < 0 || params->rule > 2)
        return sfail(SA_ERR_INVALID, "bad run parameters");
    if (params->trace || params->energy_trace || params->report || params->init_states)
        return sfail(SA_ERR_UNSUPPORTED, "served requests take no traces, report or initial states");
    if (params->rule == SA_OPT_METROPOLIS && v.max_exp > 4)
        return sfail(SA_ERR_UNSUPPORTED, "OTM needs exponents <= 4");
    Request* r = new Request();
    r->model = model;
    r->params = *params;
    if (params->temperatures) r->temps.assign(params->temperatures, params->temperatures + params->n_sweeps);
    r->n = v.n;
    r->is_float = v.is_float != 0;
    r->bytes = request_bytes(*r, v) + sa_internal_model_bytes(model);
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
    if (states) std::memcpy(states, r->h_states, R * n * 4);
    if (energies) std::memcpy(energies, r->h_en, R * 8);
    if (accepts) std::memcpy(accepts, r->h_acc, R * 8);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_end - r->t_submit).count();
    cudaFreeHost(r->h_states);
    cudaFreeHost(r->h_en);
    cudaFreeHost(r->h_acc);
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
    return SA_OK;
}

void sa_server_destroy(sa_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& kv : s->reqs)
            if (kv.second->state == SA_REQ_QUEUED) kv.second->state = SA_REQ_CANCELLED;
    }
    // let running requests finish (bounded), then stop the dispatcher
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
    for (auto& kv : s->reqs) {
        Request* r = kv.second;
        free_request_device(r, r->stream_slot >= 0 ? s->streams[r->stream_slot] : (cudaStream_t)0);
        if (r->h_states) cudaFreeHost(r->h_states);
        if (r->h_en) cudaFreeHost(r->h_en);
        if (r->h_acc) cudaFreeHost(r->h_acc);
        delete r;
    }
    for (auto& st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    delete s;
}

}  // extern "C"
