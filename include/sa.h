/*
 * sa.h -- C ABI of the GB300 (sm_103a) library for direct simulated annealing
 * (SA) on quadratic and higher-order unconstrained integer optimization
 * (QUIO / HUIO), after K. Suzuki, arXiv:2511.17245.
 *
 * The library runs the single-variable update sweep of Sect. 3 on the GPU:
 * for each integer variable in index order it evaluates the energy change of
 * a candidate value from cached per-replica coefficients (Eq. energy_diff_quad
 * for QUIO, Eq. energy_diff_poly for HUIO), draws the move by Metropolis
 * (Sect. 3.3.1), heat bath (Eq. prob_heatbath, with the O(1) inverse transform
 * of Eq. inverse_prob for multilinear variables) or optimal-transition
 * Metropolis (Eq. eq_opt_trans), and updates the cached coefficients of the
 * variables that share a term with the moved one (Eq. energy_diff_upd).
 *
 * Conventions for every entry point
 *   - Plain C types only.  `stream` is a cudaStream_t passed as void*
 *     (NULL = the legacy default stream).  All work is enqueued on it.
 *   - Pointers marked "host or device" are classified with
 *     cudaPointerGetAttributes.  When every output is device memory the call
 *     is asynchronous on `stream`; when any output is host memory the call
 *     copies through device temporaries and synchronises `stream` before it
 *     returns.
 *   - The caller owns every buffer it passes; the library copies what it needs
 *     and keeps no pointer after the call returns.  A model owns its device
 *     copy until sa_model_destroy.
 *   - Errors are returned as sa_status; nothing aborts the process.  A
 *     human-readable message for the last failing call on the calling thread
 *     is available from sa_last_error().
 *   - A model lives on the CUDA device that was current when it was created;
 *     calls that use it must run with that device current.
 */
#ifndef SA_GB300_H
#define SA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SA_OK = 0,
    SA_ERR_INVALID = 1,      /* malformed argument, bound or term list       */
    SA_ERR_OVERFLOW = 2,     /* integer model could overflow int64 (see below) */
    SA_ERR_UNSUPPORTED = 3,  /* valid request outside what the kernels cover */
    SA_ERR_OOM = 4,          /* device allocation failed                     */
    SA_ERR_CUDA = 5,         /* a CUDA runtime call or launch failed         */
    SA_ERR_TIMEOUT = 6,      /* a bounded wait gave up                       */
    SA_ERR_BUSY = 7          /* the resource is in use                       */
} sa_status;

typedef enum {
    SA_COEF_I32 = 0,         /* int32_t coefficients: exact int64 arithmetic   */
    SA_COEF_I64 = 1,         /* int64_t coefficients: exact int64 arithmetic   */
    SA_COEF_F32 = 2,         /* float coefficients: fp32 fields, FP64 refresh  */
    SA_COEF_F64 = 3          /* double coefficients: fp32 fields, FP64 refresh */
} sa_coef_type;

typedef enum {
    SA_METROPOLIS = 0,       /* Sect. 3.3.1 */
    SA_HEAT_BATH = 1,        /* Sect. 3.3.2, Eqs. prob_heatbath, inverse_prob */
    SA_OPT_METROPOLIS = 2    /* Sect. 3.3.3, Eq. eq_opt_trans */
} sa_rule;

typedef struct sa_model sa_model;   /* opaque, owned by the library */

/*
 * sa_model_create -- compile a QUIO/HUIO objective (Eqs. def_QUIO, def_HUIO)
 * into a device-resident model.
 *
 *   out           receives the new model; *out is NULL on failure.
 *   n_vars        N >= 1.
 *   lower, upper  host int64[N]: bounds l_i <= z_i <= u_i (Sect. 2).  Each
 *                 bound must fit int32 and u_i - l_i must be < 2^31.
 *   n_terms       number of terms (>= 0).
 *   term_offsets  host int64[n_terms + 1], term_offsets[0] = 0, non-decreasing:
 *                 term t is term_vars[term_offsets[t] .. term_offsets[t+1]).
 *   term_vars     host int32: each term's index multiset.  Order is irrelevant;
 *                 a repeated index is a power (z_k^m); a one-index term is a
 *                 linear term; an empty term is a constant.
 *   coeffs        host array of n_terms values of `coef_type`.
 *
 * Terms with equal multisets are merged by summing (Sect. 2); terms whose
 * merged coefficient is exactly zero are dropped.  Integer models are checked
 * against int64 overflow: with z^max_i = max(|l_i|, |u_i|, 1), the sum over
 * terms of |J| prod z^max must stay below 2^62, and for every variable k the
 * bound sum_m a~_k^(m) * 2 (z^max_k)^m (a~ as in Sect. 3.4) must stay below
 * 2^62; otherwise SA_ERR_OVERFLOW.  NaN/Inf coefficients, out-of-range indices
 * and l > u give SA_ERR_INVALID; exponents above 63 give SA_ERR_UNSUPPORTED.
 */
sa_status sa_model_create(sa_model** out, int32_t n_vars, const int64_t* lower, const int64_t* upper,
                          int64_t n_terms, const int64_t* term_offsets, const int32_t* term_vars,
                          const void* coeffs, sa_coef_type coef_type);

/*
 * sa_model_create_quio_dense -- dense QUIO (Eq. def_QUIO) from a coefficient
 * matrix: E = sum_k h_k z_k + sum_k J_kk z_k^2 + sum_{i<j} J_ij z_i z_j.
 *   h  host array of n values, J  host n x n row-major array (both of
 *   coef_type).  J is read on and above the diagonal only (a symmetric matrix
 *   counts each unordered pair once, Sect. 2); zero entries are skipped.
 * Same checks, results and model as sa_model_create with the equivalent term
 * list, without hashing n^2 terms.
 */
sa_status sa_model_create_quio_dense(sa_model** out, int32_t n_vars, const int64_t* lower, const int64_t* upper,
                                     const void* h, const void* J, sa_coef_type coef_type);

/* Releases the model and its device memory.  NULL is ignored.  The caller must
 * make sure no enqueued work still uses the model. */
void sa_model_destroy(sa_model* model);

typedef struct {
    int32_t n_vars;
    int32_t is_float;         /* 1 for SA_COEF_F32/F64 models                   */
    int32_t is_quadratic;     /* every merged term has total degree <= 2        */
    int32_t max_exponent;     /* largest power of one variable in one term      */
    int32_t max_order;        /* largest total degree of a term                 */
    int32_t all_multilinear;  /* every variable appears with exponent 1 only    */
    int64_t n_terms;          /* merged, non-zero, non-constant terms           */
    int64_t n_links;          /* QUIO: adjacency entries; HUIO: incidences      */
    int32_t n_levels;         /* dependency levels of one sweep (see run)       */
    int32_t max_width;        /* largest u_k - l_k                              */
    int64_t device_bytes;     /* device memory held by the model                */
} sa_model_info;

/* Fills `info` with a description of the compiled model. */
sa_status sa_model_get_info(const sa_model* model, sa_model_info* info);

/*
 * sa_default_temperatures -- initial and final temperature from the model
 * alone (Sect. 3.4): T_max = -dE_max / ln(1/2) with
 * dE_max ~ max_k sum_{m in Omega_k} a~_k^(m) (u_k - l_k)^m (Eq. eq_temp_init),
 * T_min = -dE_min / ln(0.001) with dE_min ~ the smallest |J| over all terms.
 * Host-only; both outputs are host pointers.
 */
sa_status sa_default_temperatures(const sa_model* model, double* t_max, double* t_min);

/* Optional per-run report, filled on the host after the run (forces a
 * synchronisation of the stream). */
typedef struct {
    double max_refresh_drift;     /* float models: max |fp32 field - FP64 field| seen at refreshes */
    int32_t replicas_per_block;   /* launch shape chosen for the sweep kernel */
    int32_t threads_per_replica;
    int32_t state_in_global;      /* 1 if the per-replica state lived in global memory */
    int32_t shared_bytes;         /* dynamic shared memory per block */
    int32_t blocks;               /* grid size of the sweep kernel */
    int32_t n_levels;
    float kernel_ms;              /* device time of the sweep kernel (CUDA events) */
    int32_t time_sliced;          /* 1 if the run was one time-sliced cooperative launch */
} sa_run_report;

/* Run flags */
#define SA_FLAG_STATE_IN_GLOBAL 0x1   /* keep per-replica state in global memory even if it fits on chip */
#define SA_FLAG_NO_TIME_SLICING 0x2   /* run more replicas than fit at once as plain waves (see sa_run) */
#define SA_FLAG_NO_SPECULATION  0x4   /* decide single-variable levels one at a time (see sa_run) */

typedef struct {
    int32_t rule;                 /* sa_rule                                              */
    int32_t n_sweeps;             /* S >= 1                                               */
    int32_t n_replicas;           /* R >= 1 independent SA runs ("samples", Sect. 4)      */
    int32_t refresh_interval;     /* float models: sweeps between FP64 refreshes; 0 -> 50 */
    uint64_t seed;                /* Philox key = (lo32(seed), hi32(seed))               */
    double t_max, t_min;          /* geometric schedule of Sect. 3.1; both <= 0 -> Sect. 3.4 defaults */
    const double* temperatures;   /* optional host double[S]: explicit T per sweep       */
    const int32_t* init_states;   /* optional int32[R][N] (host or device); else uniform random */
    uint32_t instance_id;         /* fourth Philox counter word (default 0)              */
    int32_t replicas_per_block;   /* launch shape override, 0 = automatic                */
    int32_t threads_per_replica;  /* launch shape override (multiple of 32), 0 = automatic */
    int32_t flags;                /* SA_FLAG_*                                           */
    int32_t* trace;               /* optional device int32[S][trace_replicas][N]: value of z_k after
                                     every attempt of replicas < trace_replicas (testing aid) */
    int32_t trace_replicas;
    int32_t _pad0;
    void* energy_trace;           /* optional device int64 (integer models) or double
                                     (float models) [S][R]: energy after every sweep     */
    sa_run_report* report;        /* optional host report                                */
    int32_t* best_states;         /* optional int32[R][N] (host or device): per replica, the
                                     lowest-energy state at the end of any sweep (with
                                     best_energies; see sa_run)                          */
    void* best_energies;          /* optional int64[R] (integer models) or double[R] (float
                                     models), host or device: the energy of best_states  */
} sa_run_params;

/*
 * sa_run -- R independent SA runs of Sect. 3.1 on one model.
 *
 * Random numbers: one Philox4x32-10 block per attempt with counter
 * (k, s, r, instance_id) and key (lo32(seed), hi32(seed)); the initial state
 * uses s = 0xFFFFFFFF.  U = (x >> 8) 2^-24 in [0,1), Uc = ((x >> 8) + 1) 2^-24
 * in (0,1], pick(x, M) = (x M) >> 32.  Sweep s (0-based) runs at
 * T_s = T_max (T_min/T_max)^(s/(S-1)), with beta_s = fp32(1/T_s), and OTM
 * ratio r_s = fp32(s)/fp32(S-1).
 *
 *   out_states    int32[R][N] (host or device): final z, one row per replica.
 *   out_energies  int64[R] for integer models, double[R] for float models
 *                 (host or device): final energy (exact for integer models;
 *                 FP64 recomputation from the final state for float models).
 *   out_accepts   optional uint64[R] (host or device): number of attempts that
 *                 changed the variable.
 *
 * Best-state tracking (params->best_states and params->best_energies, both
 * or neither): among the states at the ends of sweeps 0..S-1, the one with the
 * lowest tracked energy, the earliest on ties (the final state is a
 * candidate, so the best energy never exceeds the final one).  The tracked
 * energy is exact for integer models; for float models it is the fp32-updated
 * energy, exact in FP64 at refresh sweeps, and best_energies holds the FP64
 * recomputation of the chosen state.  Cost: one group reduction per sweep and
 * N int32 stores per sweep that improves on the best so far.  Not available in
 * batches, served requests and sa_run_noalloc (SA_ERR_UNSUPPORTED there).
 *
 * Visiting order: within a sweep variables are updated in index order
 * (Sect. 3.1).  The kernels run the updates of variables that share no term
 * concurrently when they form a dependency level; this reproduces the
 * sequential trajectory exactly for integer models.
 *
 * Speculative windows (QUIO): a run of levels that hold one variable each
 * (every level of a complete graph) is decided by the lanes of one warp, up
 * to 32 levels at once.  The decisions before the first one that changes its
 * variable saw the same state as in the sequential order, and so did that
 * one; its neighbours' fields are then updated and the next window starts
 * after it.  States, energies, counts and traces are those of the
 * level-by-level order, bit for bit (float models included).  Float heat bath,
 * and heat bath where a variable's range makes the kernel decide it with a
 * whole warp, keep the level-by-level order.  SA_FLAG_NO_SPECULATION disables
 * the windows.
 *
 * Time slicing: when the replicas' state stays in shared memory but more
 * replicas are requested than thread groups fit on the GPU at once, and the
 * last of the resulting waves would be less than 95% full, the run is one
 * cooperative launch in which the resident groups claim (replica, chunk of
 * about S/16 sweeps) tasks one by one; consecutive chunks of a replica pass its
 * state through a device buffer.  Results are those of the plain launch (bit
 * for bit for integer models).  SA_FLAG_NO_TIME_SLICING disables it.
 *
 * Errors: SA_ERR_INVALID for bad parameters, SA_ERR_UNSUPPORTED for OTM on a
 * variable with exponent above 4 (Sect. 3.3.3 implements degree <= 4),
 * SA_ERR_OOM / SA_ERR_CUDA for device failures.
 */
sa_status sa_run(const sa_model* model, const sa_run_params* params, int32_t* out_states,
                 void* out_energies, uint64_t* out_accepts, void* stream);

/*
 * sa_energy -- E(z) of Eq. def_HUIO for n_states states.
 *
 *   states    int32[n_states][N] (host or device), each value inside its bounds.
 *   energies  int64[n_states] for integer models, double[n_states] for float
 *             models (host or device).
 * Values outside the bounds give SA_ERR_INVALID (checked on the device; the call
 * then synchronises the stream).
 */
sa_status sa_energy(const sa_model* model, const int32_t* states, int64_t n_states, void* energies,
                    void* stream);

/*
 * Batched runs: many instances (models with their own sa_run_params) in one
 * persistent launch.  This is the replica/instance parallelism of Sect. 4
 * (independent samples) extended to independent problems; each instance's
 * results equal those of sa_run with the same parameters (same Philox counters:
 * set params[i].instance_id to keep streams distinct across instances).
 *
 * sa_batch_create  models: n_models model pointers; params: one sa_run_params
 *                  per model.  All models share one kind (QUIO or HUIO) and one
 *                  coefficient class (integer or float), and all params one rule
 *                  (SA_ERR_UNSUPPORTED otherwise).  n_sweeps, n_replicas, seed,
 *                  instance_id, temperatures and init_states (device memory) may
 *                  differ per instance; trace, best_states and best_energies must
 *                  be NULL.  The batch owns its device buffers (arguments,
 *                  schedules, outputs) and a CUDA graph holding the launch.
 *                  Synchronous.
 * sa_batch_autotune  times the launch with threads_per_replica in
 *                  {32, 64, 96, 128, 256} (replicas per block: as many as shared
 *                  memory holds) on a run truncated to trial_sweeps sweeps on
 *                  `stream`, keeps the fastest shape and re-captures the graph.
 *                  It overwrites the batch outputs.  Synchronous.
 * sa_batch_run     replays the graph on `stream` (asynchronous).
 * sa_batch_result  copies instance i's final states (int32[R_i][N_i]),
 *                  energies (int64 or double [R_i]) and change counts
 *                  (uint64[R_i]) into host or device buffers (any may be NULL);
 *                  synchronises `stream`.
 * sa_batch_destroy releases everything (NULL is ignored).
 */
typedef struct sa_batch sa_batch;
typedef struct {
    int32_t n_instances;
    int32_t n_units;              /* replicas over all instances */
    int32_t replicas_per_block;
    int32_t threads_per_replica;
    int32_t blocks;               /* persistent grid */
    int32_t state_in_global;
    int64_t attempts;             /* sum over instances of N R S */
    int64_t device_bytes;
    float autotune_ms;            /* best trial time of the last sa_batch_autotune */
    int32_t _reserved;
} sa_batch_info;
sa_status sa_batch_create(sa_batch** out, const sa_model* const* models, int32_t n_models,
                          const sa_run_params* params);
sa_status sa_batch_autotune(sa_batch* batch, int32_t trial_sweeps, void* stream);
sa_status sa_batch_run(sa_batch* batch, void* stream);
sa_status sa_batch_result(const sa_batch* batch, int32_t instance, int32_t* states, void* energies,
                          uint64_t* accepts, void* stream);
sa_status sa_batch_get_info(const sa_batch* batch, sa_batch_info* info);
void sa_batch_destroy(sa_batch* batch);

/*
 * Serving: a request loop with continuous batching.  Requests (a model and its
 * run parameters) queue in submission order; a dispatcher thread admits them,
 * skipping ahead past requests that do not fit yet, whenever a request slot is
 * free and the request's device bytes (its model plus its outputs, schedule
 * and any replica state too large for a shared-memory region) fit in
 * budget_bytes.  An admitted request's replicas become units of one device
 * work queue that a single persistent kernel drains: each of its thread groups
 * claims the next unit and runs that replica, so requests admitted while
 * others run share the GPU replica by replica, whatever their rule, model kind
 * or coefficient type.  Finished requests release their memory and slot at
 * once.  A request's results are those of sa_run with the same model and
 * parameters (bit for bit for integer models), whatever else is running.
 *
 * While admitted requests remain, the persistent kernel occupies the GPU:
 * calls that synchronise the whole device (cudaDeviceSynchronize, cudaFree,
 * sa_model_destroy) from other threads wait until the server has drained.
 *
 * sa_server_create  budget_bytes > 0; max_running in 1..8192 (requests admitted
 *                   at a time); threads_per_replica 0 (256), 64, 128 or 256:
 *                   the thread-group size of the serving kernel (two groups
 *                   of 256 per SM, each with a ~112 KB state region, by default).
 * sa_server_submit  copies params (and params->temperatures); trace,
 *                   energy_trace, report, init_states, best_states and
 *                   best_energies must be NULL.  The model
 *                   must stay alive until the request is finished.  A request
 *                   larger than the whole budget fails with SA_ERR_OOM.
 * sa_server_poll    state: SA_REQ_QUEUED, _RUNNING, _DONE, _FAILED, _CANCELLED.
 * sa_server_wait    waits at most timeout_us (SA_ERR_TIMEOUT after that).
 * sa_server_cancel  cancels a queued request (SA_ERR_BUSY once it runs).
 * sa_server_result  copies the results of a finished request into host buffers
 *                   (any may be NULL) and releases the ticket.
 * sa_server_get_stats  counts, device bytes in use and peak, attempts, p50/p99
 *                   latency (submission to completion), attempts/s from the
 *                   first submission to the last completion, finished units
 *                   and launches of the persistent kernel.
 * sa_server_destroy cancels queued requests, waits (bounded) for running ones.
 */
typedef struct sa_server sa_server;
#define SA_REQ_QUEUED 0
#define SA_REQ_RUNNING 1
#define SA_REQ_DONE 2
#define SA_REQ_FAILED 3
#define SA_REQ_CANCELLED 4
typedef struct {
    uint64_t budget_bytes;
    int32_t max_running;
    int32_t threads_per_replica;
} sa_server_config;
typedef struct {
    int64_t completed, failed, cancelled, queued, running;
    int64_t device_bytes_in_use, device_bytes_peak;
    int64_t attempts;
    double p50_latency_ms, p99_latency_ms;
    double attempts_per_s;
    int64_t units_done;           /* finished (request, replica) units */
    int64_t kernel_launches;      /* launches of the persistent serving kernel */
} sa_server_stats;
sa_status sa_server_create(sa_server** out, const sa_server_config* config);
sa_status sa_server_submit(sa_server* server, const sa_model* model, const sa_run_params* params, uint64_t* ticket);
sa_status sa_server_poll(sa_server* server, uint64_t ticket, int32_t* state);
sa_status sa_server_wait(sa_server* server, uint64_t ticket, int64_t timeout_us);
sa_status sa_server_cancel(sa_server* server, uint64_t ticket);
sa_status sa_server_result(sa_server* server, uint64_t ticket, int32_t* states, void* energies, uint64_t* accepts,
                           double* latency_ms);
sa_status sa_server_get_stats(sa_server* server, sa_server_stats* stats);
void sa_server_destroy(sa_server* server);

/*
 * sa_run_noalloc -- the run of sa_run for callers that must not allocate
 * device memory.  (The paper has no counterpart; this is a library service.)
 *
 * Who needs it: code embedded in a host framework that owns all device memory
 * through its own arena and forbids any other allocation, and latency-critical
 * callers that cannot afford an allocation (which can synchronise the device)
 * on the request path.  sa_run allocates its scratch per call; this variant
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *
 * Arguments and results are those of sa_run, with these differences:
 *   - out_states, out_energies, out_accepts and params->init_states must be
 *     device pointers (SA_ERR_INVALID otherwise); params->report must be NULL;
 *     best-state tracking is not available (SA_ERR_UNSUPPORTED).
 *   - The run's scratch (the per-sweep temperature table, and the replicas'
 *     state when it does not fit in shared memory) lives in one fixed device
 *     array of SA_NOALLOC_SCRATCH_BYTES bytes compiled into the library; every
 *     device that loads the library holds it until the process exits.  A run
 *     needing more (n_sweeps above SA_NOALLOC_SCRATCH_BYTES / 8, or replica
 *     state that must spill to global memory and does not fit beside the table)
 *     fails with SA_ERR_UNSUPPORTED and a message naming the limit.
 *   - Every call on a device shares that array and it keeps the previous call's
 *     contents; the kernel writes every scratch byte it reads.  Calls whose
 *     work overlaps on the GPU (other streams, or a new call before the last
 *     one finished on another stream) race on the array and must be serialised
 *     by the caller.
 *   - The first call on each device does a one-time set-up: with that device
 *     current it looks up the array's device address and caches it.  Make
 *     that first call before any stream capture.  The cached address belongs
 *     to the context that was current at the first call; a program that
 *     destroys that context (cudaDeviceReset) must not call sa_run_noalloc on
 *     that device afterwards.
 */
#define SA_NOALLOC_SCRATCH_BYTES (4u << 20)
sa_status sa_run_noalloc(const sa_model* model, const sa_run_params* params, int32_t* out_states,
                         void* out_energies, uint64_t* out_accepts, void* stream);

/* Message of the last failed call on the calling thread ("" if none). */
const char* sa_last_error(void);

/* Library version string. */
const char* sa_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SA_GB300_H */
