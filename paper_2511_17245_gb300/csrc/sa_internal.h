// sa_internal.h -- device model layout and kernel arguments shared by the
// host-side model compiler and launchers (api.cu, batch.cu, noalloc.cu,
// server.cu) and the CUDA kernels.
#pragma once

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
    int32_t rpc;                // replicas per block
    int32_t tpr;                // threads per replica (multiple of 32)
    int32_t heavy_links;        // link_len above which updates are cooperative
    int32_t list_cap;           // capacity of the cooperative update list
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

// Host-side launchers implemented in the .cu files.
// zbytes in {1,2,4}; returns a cudaError_t as int.
int launch_sweep(const SweepArgs& a, int zbytes, int rule, bool smem, int blocks, int threads,
                 size_t shared_bytes, void* stream);
int launch_energy(const EnergyArgs& a, void* stream);
// Persistent batched kernel; set_attr = false during stream capture.
int launch_batch(const BatchArgs& b, int is_float, int kind, int zbytes, int rule, bool smem, int blocks,
                 int threads, size_t shared_bytes, void* stream, bool set_attr);
int sweep_max_shared_optin();

}  // namespace sa
