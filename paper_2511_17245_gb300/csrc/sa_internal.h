// sa_internal.h -- device model layout and kernel arguments shared by the
// host-side model compiler and launchers (api.cu, batch.cu, noalloc.cu,
// server.cu) and the CUDA kernels.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

namespace sa {

enum Kind : int32_t { KIND_QUIO = 0, KIND_HUIO = 1 };

// Per-variable metadata, 16 bytes, read once per attempt.
struct VarMeta {
    int32_t lo;           // l_k
    uint32_t width;       // u_k - l_k (0 = fixed variable)
    int32_t link_begin;   // QUIO: first adjacency entry; HUIO: first incidence entry
    int32_t link_len;     // number of adjacency / incidence entries
};

// Per-variable record in dependency-level order, 32 bytes, everything one
// attempt needs besides the replica state.  aux holds J_kk (QUIO; fp32 bits or
// int64) or the exponent mask Omega_k (HUIO).
struct alignas(16) LevelRec {
    int32_t k;
    int32_t lo;
    uint32_t width;
    int32_t link_begin;
    int32_t link_len;
    int32_t slot_base;
    uint32_t aux0, aux1;
};

// Device-resident compiled model.  All pointers are device pointers into one
// allocation.  For integer models the *_i arrays are used; for float models
// the *_f arrays drive the sweep and the *_d arrays the FP64 refresh.
struct DevModel {
    int32_t n;
    int32_t kind;
    int32_t is_float;
    int32_t n_levels;
    uint32_t max_width;         // largest u_k - l_k
    int32_t dense_rows;         // QUIO on a complete graph: row k lists every j != k in increasing order
    const VarMeta* meta;        // [n]
    const int32_t* lvl_ptr;     // [n_levels + 1]
    const int32_t* lvl_vars;    // [n]: variables grouped by dependency level
    const LevelRec* lvl_rec;    // [n]: their records, same order

    // QUIO (every term of total degree <= 2):
    //   E = c + sum_k lin_k z_k + sum_k diag_k z_k^2 + sum_{i<j} J_ij z_i z_j
    const int32_t* adj_col;     // symmetric adjacency, both directions
    const int64_t* adj_i;
    const float* adj_f;
    const double* adj_d;        // null when the coefficients were given as fp32
    const int64_t* lin_i;
    const float* lin_f;
    const double* lin_d;
    const int64_t* diag_i;
    const float* diag_f;
    const double* diag_d;

    // HUIO: per-variable coefficient slots a_k^(m), m in Omega_k
    int32_t n_slots;
    int32_t n_iterms;           // interaction terms (two or more distinct variables)
    const int32_t* slot_base;   // [n]
    const uint64_t* omega;      // [n]: bit m set iff z_k^m appears in some term
    const int64_t* aconst_i;    // [n_slots]: single-variable terms J_{k..k} (constant part)
    const float* aconst_f;
    const double* aconst_d;
    const int32_t* inc_term;    // incidence of variable s: interaction terms containing s
    const int32_t* inc_exp;     //   and the exponent of s in that term
    // per incidence, 12 int32 (three 16-byte groups): {term, exponent of s,
    // number of other members (0..3, or -1 for terms of more than 4 members),
    // 0}, {other members' variables v1..v3, their exponents packed
    // e1 | e2 << 8 | e3 << 16}, {their coefficient slots (slot_base[v] + index
    // of the exponent), 0}
    const int32_t* inc_rec;
    const int32_t* term_ptr;    // [n_iterms + 1] into mem_var / mem_exp
    const int32_t* mem_var;     // members (distinct variables) of interaction terms
    const int32_t* mem_exp;     // their exponents
    const int64_t* tcoef_i;     // [n_iterms]
    const float* tcoef_f;
    const double* tcoef_d;

    int64_t const_i;            // empty multiset
    double const_d;
};

enum Rule : int32_t { RULE_METROPOLIS = 0, RULE_HEAT_BATH = 1, RULE_OPT = 2 };

// Arguments of the sweep kernel (passed by value).
struct SweepArgs {
    DevModel m;
    int32_t R;                  // replicas
    int32_t S;                  // sweeps
    uint32_t key0, key1;        // Philox key
    uint32_t inst;              // fourth counter word
    int32_t refresh_interval;   // float models
    const float* beta;          // [S]
    const float* ratio;         // [S]
    const int32_t* init_states; // [R][n] or null
    int32_t* out_states;        // [R][n]
    void* out_energies;         // int64 or double [R]
    unsigned long long* out_accepts;  // [R] or null
    int32_t* trace;             // [S][trace_R][n] or null
    int32_t trace_R;
    void* energy_trace;         // [S][R] or null
    unsigned int* drift_bits;   // max refresh drift (float bits, atomicMax) or null
    uint8_t* gstate;            // per-replica state slabs when not on chip
    int64_t rep_bytes;          // bytes of one replica's state region
    int32_t off_z, off_cache, off_ctl, off_list, off_red;
    int32_t off_lvl;            // level boundaries staged in the replica region (-1: read from the model)
    int32_t speculate;          // decide runs of single-variable levels a warp at a time
    int32_t _pad_spec;
    int32_t rpc;                // replicas per block
    int32_t tpr;                // threads per replica (multiple of 32)
    int32_t heavy_links;        // link_len above which updates are cooperative
    int32_t list_cap;           // capacity of the cooperative update list
    // time-sliced runs (sweep_sliced_kernel): per-replica regions through which
    // a replica's state passes from one chunk of sweeps to the next, the number
    // of finished chunks per replica, the task counter and an error word
    uint8_t* handoff;
    unsigned int* handoff_flag; // [R]: chunks of the replica finished (and saved)
    int64_t handoff_bytes;      // bytes of one region: off_ctl + 24 per thread, rounded to 16
    unsigned int* status;       // [0] bit 0: a handoff wait gave up (that replica's outputs are not
                                // written); [1]: task counter
    int32_t* best_states;       // [R][N] or null: lowest-energy state at a sweep end
    void* best_energies;        // [R] (int64 or double): its tracked energy
};

// One unit of batched work: one replica of one instance.
struct BatchUnit {
    int32_t inst;
    int32_t replica;
};

// Arguments of the persistent batched kernel.
struct BatchArgs {
    const SweepArgs* insts;     // per-instance arguments (device table)
    const BatchUnit* units;     // ordered by decreasing cost
    int32_t n_units;
    unsigned int* counter;      // next unit (reset to 0 before every launch)
    int64_t slot_bytes;         // state region of one thread group (max over instances)
    int32_t rpc, tpr;
    uint8_t* gstate;            // per-group regions when the state is not on chip
};

// ------------------------------------------------------------------ serving
// One admitted request of the server: the kernel arguments of its run (the
// fields of SweepArgs, with the layout for the serving kernel's group size)
// and which compiled variant runs it.  Written by the host into host-mapped
// memory before the request's units are published.
struct ServeReq {
    SweepArgs args;
    int32_t variant;            // serve_variant(...)
    int32_t n_units;            // replicas
};

// A unit of serving work: one replica of one admitted request.
struct ServeUnit {
    int32_t req;                // request slot
    int32_t replica;
};

// Host-mapped control words of the serving queue.
struct ServeCtl {
    volatile uint32_t tail;     // units published so far (host writes)
    volatile uint32_t stop;     // nonzero: groups leave once the queue is empty
};

// Arguments of the persistent serving kernel.
struct ServeArgs {
    const ServeReq* reqs;       // [max_reqs], host-mapped
    const ServeUnit* units;     // ring of `cap` units, host-mapped
    const ServeCtl* ctl;        // host-mapped
    unsigned int* head;         // device: next unit to claim
    unsigned int* req_units_done;   // device: [max_reqs] finished units per request slot
    unsigned int* req_done;     // host-mapped: [max_reqs] set to 1 when a request's last unit finished
    uint32_t cap;               // ring capacity (a power of two)
    int32_t tpr, rpc;
    int32_t _pad0;
    int64_t slot_bytes;         // shared-memory state region of one thread group
    uint32_t idle_polls;        // empty-queue polls (about 2 us each) before a group leaves
    uint32_t _pad1;
};

// Variant index of a request for the serving kernel: rule, model kind,
// coefficient class and 2- or 4-byte state offsets.
inline int serve_variant(int rule, int kind, int is_float, int zbytes) {
    return rule + 3 * (kind + 2 * (is_float + 2 * (zbytes > 2 ? 1 : 0)));
}

// Arguments of the energy kernel.
struct EnergyArgs {
    DevModel m;
    const int32_t* states;      // [n_states][n]
    int64_t n_states;
    void* energies;             // int64 or double
    int32_t* bad;               // set to 1 if a value lies outside its bounds
};

// Read-only view of a compiled model for translation units other than api.cu.
struct ModelView {
    DevModel dm;
    int device;
    int32_t n;
    int is_float;
    int max_exp;
    int zbytes;
    int64_t cache_elems;
    int32_t n_levels;
    int32_t max_link_len;       // longest neighbour / incidence list
    double de_max, de_min;
};

// Threads per replica for a launch whose caller left the choice to the library.
// `tpr` is the choice from the level widths; when the block's replicas leave
// thread slots unused (few replicas per SM) and some variable's update list is
// longer than `heavy_links` (the lists the whole group updates together), the
// spare slots go to the replicas.  Integer results do not depend on the shape.
inline int grow_threads_per_replica(int tpr, int32_t max_link_len, int heavy_links, int replicas,
                                    int replicas_per_block, int sms) {
    if (max_link_len <= heavy_links) return tpr;
    int per_block = replicas_per_block > 0 ? replicas_per_block : (replicas + sms - 1) / (sms > 0 ? sms : 1);
    per_block = per_block < 1 ? 1 : (per_block > 15 ? 15 : per_block);
    int grown = (512 / per_block) / 32 * 32;
    if (grown > 256) grown = 256;
    return grown > tpr ? grown : tpr;
}

// ------------------------------------------------------------------ run planning
// Host-side planning shared by every entry point that launches the sweep
// kernel (sa_run, sa_run_noalloc, batches).  Pure arithmetic: no CUDA calls,
// so that the same rules can be checked on a machine without a GPU.

// What the planner needs to know about a compiled model.
struct PlanModel {
    int32_t n;
    int32_t n_levels;
    int32_t kind;               // KIND_QUIO / KIND_HUIO
    int32_t is_float;
    int32_t zbytes;             // bytes of one state offset z_k - l_k
    int32_t max_link_len;
    int64_t cache_elems;        // QUIO: n fields; HUIO: coefficient slots
};

inline PlanModel plan_model(const ModelView& v) {
    return PlanModel{v.n, v.n_levels, v.dm.kind, v.is_float, v.zbytes, v.max_link_len, v.cache_elems};
}

// Per-replica state layout and launch shape of one run.
struct RunPlan {
    int32_t tpr;                // threads per replica (whole warps)
    int32_t rpc;                // replicas per block
    int32_t blocks;
    int32_t heavy_links;        // update lists above this length go to the cooperative list
    int32_t list_cap;           // entries of the cooperative list (6 ints each)
    int32_t in_global;          // replica state in global memory instead of shared memory
    int64_t rep_bytes;          // bytes of one replica's state region
    int64_t shared_bytes;       // dynamic shared memory of one block
    int32_t off_z, off_cache, off_ctl, off_list, off_red, off_lvl;
};

inline int64_t plan_round16(int64_t x) { return (x + 15) / 16 * 16; }

// State layout of one replica for `tpr` threads: offsets z_k - l_k (zbytes
// each), the cache (int64 or fp32), the control words (three list counters,
// the flattened length and two 48-byte results of speculative windows), the
// cooperative update list, the reduction scratch (one 8-byte word
// per warp) and, when it takes at most 16 KB, the level boundary table.
// `zbytes` may exceed the model's own (a batch uses its widest).  QUIO rows are
// cheap per entry (one atomic) and go inline up to 64 links; HUIO incidences
// cost a term product each and go inline up to 8.
inline int64_t plan_layout(const PlanModel& m, int zbytes, int tpr, RunPlan* p) {
    const bool huio = m.kind == KIND_HUIO;
    const int64_t fsize = m.is_float ? 4 : 8;
    p->tpr = tpr;
    p->heavy_links = huio ? 8 : 64;
    p->list_cap = huio ? 256 : 64;
    p->off_z = 0;
    p->off_cache = (int32_t)plan_round16((int64_t)m.n * zbytes);
    p->off_ctl = (int32_t)plan_round16(p->off_cache + m.cache_elems * fsize);
    p->off_list = p->off_ctl + 112;
    p->off_red = (int32_t)plan_round16(p->off_list + (int64_t)p->list_cap * 24);
    const int64_t lvl_bytes = (int64_t)(m.n_levels + 1) * 4;
    const int64_t off_lvl = plan_round16(p->off_red + (int64_t)(tpr / 32) * 8);
    const bool lvl_on_chip = lvl_bytes <= 16384;
    p->off_lvl = lvl_on_chip ? (int32_t)off_lvl : -1;
    p->rep_bytes = plan_round16(off_lvl + (lvl_on_chip ? lvl_bytes : 0));
    return p->rep_bytes;
}

// Launch shape of a single-model run of R replicas.  tpr_req / rpc_req <= 0
// leave the choice to the library: tpr from the mean level width (half of it,
// rounded up to whole warps, 32..256), grown by grow_threads_per_replica for
// long update lists; rpc as many replicas as shared memory and 512 threads
// allow, but no more than needed to spread the replicas over the SMs.  Returns
// nullptr, or a message describing the invalid request.
inline const char* plan_run_shape(const PlanModel& m, int32_t R, int32_t tpr_req, int32_t rpc_req, bool force_global,
                                  int sms, int64_t smem_max, RunPlan* p) {
    int tpr = tpr_req;
    if (tpr <= 0) {
        const double mean_w = (double)m.n / (double)(m.n_levels > 0 ? m.n_levels : 1);
        int want = (int)(mean_w / 2.0);
        if ((double)want < mean_w / 2.0) ++want;
        tpr = (want + 31) / 32 * 32;
        tpr = tpr < 32 ? 32 : (tpr > 256 ? 256 : tpr);
    }
    if (tpr % 32 != 0 || tpr > 512 || tpr < 32) return "threads_per_replica must be a multiple of 32, <= 512";
    if (tpr_req <= 0)
        tpr = grow_threads_per_replica(tpr, m.max_link_len, m.kind == KIND_HUIO ? 8 : 64, R, rpc_req, sms);
    const int64_t rep = plan_layout(m, m.zbytes, tpr, p);
    int fit = (int)(smem_max / rep);
    const int cap = 15 < 512 / tpr ? 15 : 512 / tpr;
    fit = fit < cap ? fit : cap;
    const bool in_global = fit < 1 || force_global;
    int rpc = rpc_req;
    if (rpc <= 0) {
        int target = (R + (sms > 0 ? sms : 1) - 1) / (sms > 0 ? sms : 1);
        target = target < 1 ? 1 : target;
        rpc = in_global ? (target < cap ? target : cap) : (fit < target ? fit : target);
    }
    if (rpc < 1 || rpc > 15 || rpc * tpr > 512) return "replicas_per_block out of range";
    if (!in_global && rpc > fit) return "replicas_per_block exceeds shared memory";
    p->rpc = rpc;
    p->in_global = in_global ? 1 : 0;
    p->blocks = (R + rpc - 1) / rpc;
    p->shared_bytes = in_global ? 0 : (int64_t)rpc * rep;
    return nullptr;
}

// ------------------------------------------------------------------ time-sliced runs
// When R replicas exceed the P thread groups that can be resident at once, a
// plain launch runs ceil(R / P) waves and the last one leaves slots idle.  A
// time-sliced launch instead cuts every replica's S sweeps into C chunks of K
// sweeps and lets the resident groups claim (replica, chunk) tasks from one
// counter in chunk-major order: task q is chunk q / R of replica q % R.  A
// chunk after the first waits for its replica's previous chunk, restores the
// state that chunk saved and saves its own for the next.  Every task's
// predecessor was claimed earlier by a resident group, so the chain of waits
// always ends at a running task; and with R >= P a predecessor was claimed
// about R tasks earlier, so it has usually finished.  Claiming tasks one by one
// balances the groups by the actual cost of the sweeps (which varies along the
// schedule), the last round of tasks being one chunk long.
constexpr int kSliceChunks = 16;

// Sweeps per chunk of a time-sliced run of S sweeps (at most kSliceChunks chunks).
inline
#ifdef __CUDACC__
__host__ __device__
#endif
int32_t slice_chunk_sweeps(int32_t S) {
    return (S + kSliceChunks - 1) / kSliceChunks;
}

// Per-sweep table read by the kernel: tab[s] = fp32(1 / T_s) with the geometric
// schedule T_s = T_max (T_min / T_max)^(s / (S - 1)) of Sect. 3.1 (T_0 = T_max
// when S = 1) or the caller's temperatures, and tab[S + s] = the OTM ratio
// r_s = fp32(s) / fp32(S - 1) of Sect. 3.3.3 (0 when S = 1).  t_max and t_min
// both <= 0 select the Sect. 3.4 temperatures -dE_max / ln(1/2) and
// -dE_min / ln(0.001).  Returns nullptr or an error message.
inline const char* plan_schedule(double de_max, double de_min, int32_t S, double t_max, double t_min,
                                 const double* temps, float* tab) {
    if (!temps) {
        if (t_max <= 0 && t_min <= 0) {
            t_max = -de_max / std::log(0.5);
            t_min = -de_min / std::log(0.001);
        } else if (!(t_max > 0 && t_min > 0) || !std::isfinite(t_max) || !std::isfinite(t_min)) {
            return "t_max and t_min must both be positive (or both <= 0 for defaults)";
        }
    }
    for (int32_t s = 0; s < S; ++s) {
        double T;
        if (temps) {
            T = temps[s];
            if (!(T > 0) || !std::isfinite(T)) return "temperatures must be positive";
        } else {
            const double frac = S > 1 ? (double)s / (double)(S - 1) : 0.0;
            T = t_max * std::pow(t_min / t_max, frac);
        }
        tab[s] = (float)(1.0 / T);
        tab[S + s] = S > 1 ? (float)s / (float)(S - 1) : 0.0f;
    }
    return nullptr;
}

// Copies the layout and shape of a plan into the kernel arguments.
inline void plan_apply(const RunPlan& p, SweepArgs& a) {
    a.rep_bytes = p.rep_bytes;
    a.off_z = p.off_z;
    a.off_cache = p.off_cache;
    a.off_ctl = p.off_ctl;
    a.off_list = p.off_list;
    a.off_red = p.off_red;
    a.off_lvl = p.off_lvl;
    a.rpc = p.rpc;
    a.tpr = p.tpr;
    a.heavy_links = p.heavy_links;
    a.list_cap = p.list_cap;
}

// Host-side launchers implemented in the .cu files.
// zbytes in {1,2,4}; returns a cudaError_t as int.
int launch_sweep(const SweepArgs& a, int zbytes, int rule, bool smem, int blocks, int threads,
                 size_t shared_bytes, void* stream);
int launch_energy(const EnergyArgs& a, void* stream);
// Time-sliced cooperative launch of `grid` blocks (state in shared memory);
// with grid = 0 it only reports the resident blocks per SM in *blocks_per_sm.
int launch_sweep_sliced(const SweepArgs& a, int zbytes, int rule, int grid, int threads, size_t shared_bytes,
                        void* stream, int* blocks_per_sm);
// Persistent batched kernel; set_attr = false during stream capture.
int launch_batch(const BatchArgs& b, int is_float, int kind, int zbytes, int rule, bool smem, int blocks,
                 int threads, size_t shared_bytes, void* stream, bool set_attr);
int sweep_max_shared_optin();
// Persistent serving kernel (blocks of rpc * tpr threads; grid = 0 only sets
// the shared-memory attribute); returns a cudaError_t as int.
int launch_serve(const ServeArgs& s, int grid, size_t shared_bytes, void* stream);
// Static shared memory of the serving kernel (per block).
size_t serve_static_shared();

}  // namespace sa
