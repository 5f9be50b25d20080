// api.cu -- host side of the C ABI declared in include/sa.h: model compilation
// (merging, classification, device layout, dependency levels, int64 overflow
// bounds, default temperatures) and the run / energy entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "sa.h"
#include "sa_internal.h"

using sa::DevModel;
using sa::VarMeta;

namespace {

thread_local std::string g_last_error;

sa_status fail(sa_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

sa_status cuda_fail(cudaError_t e, const char* where) {
    return fail(e == cudaErrorMemoryAllocation ? SA_ERR_OOM : SA_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// saturating unsigned 128-bit arithmetic for the overflow bound
typedef unsigned __int128 u128;
const u128 kSat = (u128)1 << 100;
u128 sat_mul(u128 a, u128 b) {
    if (a == 0 || b == 0) return 0;
    if (a > kSat / b) return kSat;
    u128 r = a * b;
    return r > kSat ? kSat : r;
}
u128 sat_add(u128 a, u128 b) {
    u128 r = a + b;
    return r > kSat ? kSat : r;
}

struct Member {
    int32_t var;
    int32_t exp;
};

// View of a term's members inside a shared pool.
struct MSpan {
    const Member* p = nullptr;
    size_t n = 0;
    const Member* begin() const { return p; }
    const Member* end() const { return p + n; }
    size_t size() const { return n; }
    const Member& operator[](size_t i) const { return p[i]; }
};

struct MergedTerm {
    int64_t moff = 0;         // first member in the pool
    int32_t nmem = 0;
    MSpan mem;                // distinct variables, sorted (set once the pool is final)
    __int128 ci;
    double cf;
    int order() const {
        int o = 0;
        for (auto& x : mem) o += x.exp;
        return o;
    }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct sa_model {
    int device = 0;
    DevModel dm{};
    void* dmem = nullptr;
    size_t dbytes = 0;
    int32_t n = 0;
    bool is_float = false;
    bool quadratic = false;
    bool multilinear = false;
    int max_exp = 0;
    int max_order = 0;
    int64_t n_terms = 0;
    int64_t n_links = 0;
    int32_t n_levels = 0;
    uint32_t max_width = 0;
    int zbytes = 1;
    int64_t cache_elems = 0;
    int32_t max_link_len = 0;
    double de_max = 0.0, de_min = 0.0;
    bool f32_coeffs = false;   // coefficients given as fp32: the FP64 refresh promotes the fp32 values
};

namespace {

// ------------------------------------------------------------------ device blob builder
struct Blob {
    std::vector<uint8_t> host;
    template <class T>
    size_t add(const std::vector<T>& v) {
        size_t off = align_up(host.size(), 256);
        host.resize(off + std::max<size_t>(v.size() * sizeof(T), 16));
        if (!v.empty()) std::memcpy(host.data() + off, v.data(), v.size() * sizeof(T));
        return off;
    }
};

template <class T>
const T* at(void* base, size_t off) {
    return reinterpret_cast<const T*>(static_cast<uint8_t*>(base) + off);
}

// dependency levels of the sequential sweep: level(k) = 1 + max level of the
// neighbours j < k (0 if none); neighbours share a term with k.
void build_levels(int32_t n, const std::vector<int64_t>& nb_ptr, const std::vector<int32_t>& nb,
                  std::vector<int32_t>& lvl_ptr, std::vector<int32_t>& lvl_vars, int32_t& n_levels) {
    std::vector<int32_t> level(n, 0);
    int32_t mx = 0;
    for (int32_t k = 0; k < n; ++k) {
        int32_t l = 0;
        for (int64_t e = nb_ptr[k]; e < nb_ptr[k + 1]; ++e) {
            const int32_t j = nb[e];
            if (j < k) l = std::max(l, level[j] + 1);
        }
        level[k] = l;
        mx = std::max(mx, l);
    }
    n_levels = mx + 1;
    lvl_ptr.assign(n_levels + 1, 0);
    for (int32_t k = 0; k < n; ++k) lvl_ptr[level[k] + 1]++;
    for (int32_t l = 0; l < n_levels; ++l) lvl_ptr[l + 1] += lvl_ptr[l];
    lvl_vars.assign(n, 0);
    std::vector<int32_t> fill(lvl_ptr.begin(), lvl_ptr.end() - 1);
    for (int32_t k = 0; k < n; ++k) lvl_vars[fill[level[k]]++] = k;
}

// Second half of model compilation, shared by the term-list and dense entry
// points: drops zero terms, classifies, checks the int64 bounds, derives the
// Sect. 3.4 temperatures and lays the model out on the device.
sa_status compile_terms(sa_model* M, int32_t n, const int64_t* lower, const int64_t* upper,
                        const std::vector<int32_t>& lo, const std::vector<uint32_t>& width,
                        std::vector<MergedTerm>& terms, std::vector<Member>& pool, __int128 const_i, double const_d) {
    for (auto& t : terms) t.mem = MSpan{pool.data() + t.moff, (size_t)t.nmem};
    // drop zero terms
    std::vector<MergedTerm> kept;
    kept.reserve(terms.size());
    for (auto& t : terms) {
        const bool zero = M->is_float ? (t.cf == 0.0) : (t.ci == 0);
        if (!zero) kept.push_back(std::move(t));
    }
    terms.swap(kept);
    for (auto& t : terms) {
        if (!M->is_float && (t.ci > (__int128)INT64_MAX || t.ci < (__int128)INT64_MIN))
            return fail(SA_ERR_OVERFLOW, "merged coefficient does not fit int64");
        for (auto& m : t.mem)
            if (m.exp > 63) return fail(SA_ERR_UNSUPPORTED, "exponent above 63");
    }
    if (!M->is_float && (const_i > (__int128)INT64_MAX || const_i < (__int128)INT64_MIN))
        return fail(SA_ERR_OVERFLOW, "constant term does not fit int64");
    M->n_terms = (int64_t)terms.size();

    // ---- classification
    bool quadratic = true, multilinear = true;
    int max_exp = 0, max_order = 0;
    for (auto& t : terms) {
        const int o = t.order();
        max_order = std::max(max_order, o);
        if (o > 2) quadratic = false;
        for (auto& m : t.mem) {
            max_exp = std::max(max_exp, (int)m.exp);
            if (m.exp > 1) multilinear = false;
        }
    }
    M->quadratic = quadratic;
    M->multilinear = multilinear;
    M->max_exp = max_exp;
    M->max_order = max_order;

    // ---- int64 overflow bound (integer models)
    std::vector<u128> zmax(n);
    for (int32_t k = 0; k < n; ++k) {
        const int64_t a = std::llabs(lower[k]), b = std::llabs(upper[k]);
        zmax[k] = (u128)std::max<int64_t>(1, std::max(a, b));
    }
    // per-variable a~ (Sect. 3.4) and dE_min for default temperatures
    std::vector<double> de_var(n, 0.0);
    double de_min = INFINITY;
    {
        u128 ebound = 0;
        std::vector<u128> vbound(n, 0);
        for (auto& t : terms) {
            const double absj = M->is_float ? std::fabs(t.cf) : std::fabs((double)t.ci);
            if (absj > 0 && absj < de_min) de_min = absj;
            if (!M->is_float) {
                u128 b = (u128)(t.ci < 0 ? -t.ci : t.ci);
                for (auto& m : t.mem)
                    for (int e = 0; e < m.exp; ++e) b = sat_mul(b, zmax[m.var]);
                ebound = sat_add(ebound, b);
                for (auto& m : t.mem) vbound[m.var] = sat_add(vbound[m.var], sat_mul(b, 2));
            }
            // dE_max contribution: |J| prod_{i != k} z^max_i^{e_i} (u_k - l_k)^{e_k}
            for (auto& mk : t.mem) {
                double c = absj;
                for (auto& mi : t.mem) {
                    if (mi.var == mk.var) continue;
                    const double zm = std::max(std::fabs((double)lower[mi.var]), std::fabs((double)upper[mi.var]));
                    c *= std::pow(zm, (double)mi.exp);
                }
                c *= std::pow((double)width[mk.var], (double)mk.exp);
                de_var[mk.var] += c;
            }
        }
        if (!M->is_float) {
            const u128 lim = (u128)1 << 62;
            if (ebound >= lim) return fail(SA_ERR_OVERFLOW, "energy bound sum |J| prod z^max reaches 2^62");
            for (int32_t k = 0; k < n; ++k)
                if (vbound[k] >= lim)
                    return fail(SA_ERR_OVERFLOW, "energy-difference bound reaches 2^62 at variable " + std::to_string(k));
        }
    }
    double de_max = 0.0;
    for (int32_t k = 0; k < n; ++k) de_max = std::max(de_max, de_var[k]);
    if (!std::isfinite(de_min)) de_min = 1.0;
    if (de_max <= 0.0) de_max = de_min;
    M->de_max = de_max;
    M->de_min = de_min;
    M->zbytes = M->max_width <= 0xFFu ? 1 : (M->max_width <= 0xFFFFu ? 2 : 4);

    // ---- device layout
    Blob blob;
    std::vector<VarMeta> meta(n);
    std::vector<int64_t> nb_ptr(n + 1, 0);
    std::vector<int32_t> nb;
    DevModel& dm = M->dm;
    dm.n = n;
    dm.is_float = M->is_float ? 1 : 0;
    dm.max_width = M->max_width;
    dm.const_i = (int64_t)const_i;
    dm.const_d = const_d;
    struct Offs {
        size_t meta, lvl_ptr, lvl_vars, lvl_rec;
        size_t adj_col, adj_i, adj_f, adj_d, lin_i, lin_f, lin_d, diag_i, diag_f, diag_d;
        size_t slot_base, omega, aconst_i, aconst_f, aconst_d, inc_term, inc_exp, inc_rec, term_ptr, mem_var, mem_exp,
            tcoef_i, tcoef_f, tcoef_d;
    } off{};
    std::vector<int32_t> lvl_ptr, lvl_vars;

    if (quadratic) {
        dm.kind = sa::KIND_QUIO;
        std::vector<int64_t> lin_i(n, 0), diag_i(n, 0);
        std::vector<double> lin_d(n, 0.0), diag_d(n, 0.0);
        std::vector<int64_t> deg(n, 0);
        for (auto& t : terms) {
            if (t.mem.size() == 2) {
                deg[t.mem[0].var]++;
                deg[t.mem[1].var]++;
            }
        }
        // rows padded to multiples of 4 entries (16-byte aligned starts for
        // vector loads); padding entries are never read as entries
        std::vector<int64_t> ptr(n + 1, 0);
        for (int32_t k = 0; k < n; ++k) ptr[k + 1] = ptr[k] + (deg[k] + 3) / 4 * 4;
        std::vector<int32_t> col(ptr[n], 0);
        std::vector<int64_t> vi(ptr[n], 0);
        std::vector<double> vd(ptr[n], 0.0);
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (auto& t : terms) {
            if (t.mem.size() == 1) {
                const int32_t k = t.mem[0].var;
                if (t.mem[0].exp == 1) { lin_i[k] += (int64_t)t.ci; lin_d[k] += t.cf; }
                else { diag_i[k] += (int64_t)t.ci; diag_d[k] += t.cf; }
            } else {
                const int32_t a = t.mem[0].var, b = t.mem[1].var;
                col[fill[a]] = b; vi[fill[a]] = (int64_t)t.ci; vd[fill[a]] = t.cf; fill[a]++;
                col[fill[b]] = a; vi[fill[b]] = (int64_t)t.ci; vd[fill[b]] = t.cf; fill[b]++;
            }
        }
        // sort each row by column for locality
        for (int32_t k = 0; k < n; ++k) {
            if (std::is_sorted(col.begin() + ptr[k], col.begin() + ptr[k] + deg[k])) continue;
            std::vector<int64_t> order(deg[k]);
            for (size_t i = 0; i < order.size(); ++i) order[i] = ptr[k] + (int64_t)i;
            std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return col[x] < col[y]; });
            std::vector<int32_t> c2(order.size());
            std::vector<int64_t> i2(order.size());
            std::vector<double> d2(order.size());
            for (size_t i = 0; i < order.size(); ++i) { c2[i] = col[order[i]]; i2[i] = vi[order[i]]; d2[i] = vd[order[i]]; }
            for (size_t i = 0; i < order.size(); ++i) { col[ptr[k] + i] = c2[i]; vi[ptr[k] + i] = i2[i]; vd[ptr[k] + i] = d2[i]; }
        }
        if (ptr[n] > INT32_MAX) return fail(SA_ERR_UNSUPPORTED, "more than 2^31 adjacency entries");
        for (int32_t k = 0; k < n; ++k) {
            meta[k] = {lo[k], width[k], (int32_t)ptr[k], (int32_t)deg[k]};
            M->max_link_len = std::max(M->max_link_len, meta[k].link_len);
        }
        M->n_links = 0;
        for (int32_t k = 0; k < n; ++k) M->n_links += deg[k];
        // complete graph: rows are sorted, so row k lists 0..k-1, k+1..n-1
        dm.dense_rows = 1;
        for (int32_t k = 0; k < n && dm.dense_rows; ++k)
            if (deg[k] != n - 1) dm.dense_rows = 0;
        // neighbour lists for the levels (without padding)
        nb_ptr.assign(n + 1, 0);
        for (int32_t k = 0; k < n; ++k) nb_ptr[k + 1] = nb_ptr[k] + deg[k];
        nb.resize(nb_ptr[n]);
        for (int32_t k = 0; k < n; ++k)
            for (int64_t i = 0; i < deg[k]; ++i) nb[nb_ptr[k] + i] = col[ptr[k] + i];
        build_levels(n, nb_ptr, nb, lvl_ptr, lvl_vars, M->n_levels);
        // Variables of one level are independent, so their order inside the
        // level is free.  Sorting by (J_kk, u_k - l_k) puts variables whose
        // heat-bath windows have similar widths into the same warp.
        for (int32_t L = 0; L < M->n_levels; ++L) {
            auto b = lvl_vars.begin() + lvl_ptr[L], e = lvl_vars.begin() + lvl_ptr[L + 1];
            std::stable_sort(b, e, [&](int32_t x, int32_t y) {
                const double dx = M->is_float ? diag_d[x] : (double)diag_i[x];
                const double dy = M->is_float ? diag_d[y] : (double)diag_i[y];
                if (dx != dy) return dx > dy;
                return width[x] > width[y];
            });
        }
        std::vector<sa::LevelRec> rec(n);
        for (int32_t i = 0; i < n; ++i) {
            const int32_t k = lvl_vars[i];
            sa::LevelRec& q = rec[i];
            q.k = k;
            q.lo = meta[k].lo;
            q.width = meta[k].width;
            q.link_begin = meta[k].link_begin;
            q.link_len = meta[k].link_len;
            q.slot_base = 0;
            if (M->is_float) {
                const float dv = (float)diag_d[k];
                std::memcpy(&q.aux0, &dv, 4);
                q.aux1 = 0;
            } else {
                const uint64_t dv = (uint64_t)diag_i[k];
                q.aux0 = (uint32_t)dv;
                q.aux1 = (uint32_t)(dv >> 32);
            }
        }
        off.meta = blob.add(meta);
        off.lvl_ptr = blob.add(lvl_ptr);
        off.lvl_vars = blob.add(lvl_vars);
        off.lvl_rec = blob.add(rec);
        off.adj_col = blob.add(col);
        if (M->is_float) {
            std::vector<float> vf(vd.size()), lf(n), df(n);
            for (size_t i = 0; i < vd.size(); ++i) vf[i] = (float)vd[i];
            for (int32_t k = 0; k < n; ++k) { lf[k] = (float)lin_d[k]; df[k] = (float)diag_d[k]; }
            off.adj_f = blob.add(vf);
            off.adj_d = M->f32_coeffs ? SIZE_MAX : blob.add(vd);
            off.lin_f = blob.add(lf); off.lin_d = blob.add(lin_d);
            off.diag_f = blob.add(df); off.diag_d = blob.add(diag_d);
        } else {
            off.adj_i = blob.add(vi); off.lin_i = blob.add(lin_i); off.diag_i = blob.add(diag_i);
        }
        M->cache_elems = n;
    } else {
        dm.kind = sa::KIND_HUIO;
        // exponent sets Omega_k and slot bases
        std::vector<uint64_t> omega(n, 0);
        for (auto& t : terms)
            for (auto& m : t.mem) omega[m.var] |= (1ull << m.exp);
        std::vector<int32_t> slot_base(n + 1, 0);
        for (int32_t k = 0; k < n; ++k) slot_base[k + 1] = slot_base[k] + __builtin_popcountll(omega[k]);
        const int32_t n_slots = slot_base[n];
        auto slot_of = [&](int32_t k, int32_t e) {
            return slot_base[k] + __builtin_popcountll((omega[k] & ((1ull << e) - 1ull)) >> 1);
        };
        std::vector<int64_t> aconst_i(n_slots, 0);
        std::vector<double> aconst_d(n_slots, 0.0);
        // interaction terms
        std::vector<int32_t> term_ptr(1, 0), mem_var, mem_exp;
        std::vector<int64_t> tcoef_i;
        std::vector<double> tcoef_d;
        std::vector<int64_t> ninc(n, 0);
        for (auto& t : terms) {
            if (t.mem.size() == 1) {
                const int32_t s = slot_of(t.mem[0].var, t.mem[0].exp);
                aconst_i[s] += (int64_t)t.ci;
                aconst_d[s] += t.cf;
                continue;
            }
            for (auto& m : t.mem) {
                mem_var.push_back(m.var);
                mem_exp.push_back(m.exp);
                ninc[m.var]++;
            }
            term_ptr.push_back((int32_t)mem_var.size());
            tcoef_i.push_back((int64_t)t.ci);
            tcoef_d.push_back(t.cf);
        }
        const int32_t n_iterms = (int32_t)tcoef_i.size();
        std::vector<int64_t> iptr(n + 1, 0);
        for (int32_t k = 0; k < n; ++k) iptr[k + 1] = iptr[k] + ninc[k];
        if (iptr[n] > INT32_MAX) return fail(SA_ERR_UNSUPPORTED, "more than 2^31 incidences");
        std::vector<int32_t> inc_term(iptr[n]), inc_exp(iptr[n]);
        std::vector<int64_t> fill(iptr.begin(), iptr.end() - 1);
        for (int32_t tt = 0; tt < n_iterms; ++tt)
            for (int32_t p = term_ptr[tt]; p < term_ptr[tt + 1]; ++p) {
                const int32_t v = mem_var[p];
                inc_term[fill[v]] = tt;
                inc_exp[fill[v]] = mem_exp[p];
                fill[v]++;
            }
        for (int32_t k = 0; k < n; ++k) {
            meta[k] = {lo[k], width[k], (int32_t)iptr[k], (int32_t)(iptr[k + 1] - iptr[k])};
            M->max_link_len = std::max(M->max_link_len, meta[k].link_len);
        }
        M->n_links = iptr[n];
        // incidence records: everything one cache update of Eq. energy_diff_upd
        // needs for a term of at most 4 members, read in one step
        std::vector<int32_t> inc_rec((size_t)iptr[n] * 12, 0);
        for (int32_t k = 0; k < n; ++k)
            for (int64_t e = iptr[k]; e < iptr[k + 1]; ++e) {
                int32_t* q = inc_rec.data() + (size_t)e * 12;
                const int32_t tt = inc_term[e];
                const int32_t nm = term_ptr[tt + 1] - term_ptr[tt];
                q[0] = tt;
                q[1] = inc_exp[e];
                if (nm > 4) {
                    q[2] = -1;
                    continue;
                }
                int c = 0, packed = 0;
                for (int32_t p = term_ptr[tt]; p < term_ptr[tt + 1]; ++p) {
                    const int32_t v = mem_var[p];
                    if (v == k) continue;
                    q[4 + c] = v;
                    packed |= mem_exp[p] << (8 * c);
                    q[8 + c] = slot_of(v, mem_exp[p]);
                    ++c;
                }
                q[2] = c;
                q[7] = packed;
            }
        // neighbours for levels: members of incident interaction terms
        nb_ptr.assign(n + 1, 0);
        for (int32_t k = 0; k < n; ++k) {
            int64_t c = 0;
            for (int64_t e = iptr[k]; e < iptr[k + 1]; ++e) c += term_ptr[inc_term[e] + 1] - term_ptr[inc_term[e]] - 1;
            nb_ptr[k + 1] = nb_ptr[k] + c;
        }
        nb.resize(nb_ptr[n]);
        for (int32_t k = 0; k < n; ++k) {
            int64_t w = nb_ptr[k];
            for (int64_t e = iptr[k]; e < iptr[k + 1]; ++e) {
                const int32_t tt = inc_term[e];
                for (int32_t p = term_ptr[tt]; p < term_ptr[tt + 1]; ++p)
                    if (mem_var[p] != k) nb[w++] = mem_var[p];
            }
        }
        build_levels(n, nb_ptr, nb, lvl_ptr, lvl_vars, M->n_levels);
        slot_base.resize(n);
        std::vector<sa::LevelRec> rec(n);
        for (int32_t i = 0; i < n; ++i) {
            const int32_t k = lvl_vars[i];
            sa::LevelRec& q = rec[i];
            q.k = k;
            q.lo = meta[k].lo;
            q.width = meta[k].width;
            q.link_begin = meta[k].link_begin;
            q.link_len = meta[k].link_len;
            q.slot_base = slot_base[k];
            q.aux0 = (uint32_t)omega[k];
            q.aux1 = (uint32_t)(omega[k] >> 32);
        }
        off.meta = blob.add(meta);
        off.lvl_ptr = blob.add(lvl_ptr);
        off.lvl_vars = blob.add(lvl_vars);
        off.lvl_rec = blob.add(rec);
        off.slot_base = blob.add(slot_base);
        off.omega = blob.add(omega);
        off.inc_term = blob.add(inc_term);
        off.inc_exp = blob.add(inc_exp);
        off.inc_rec = blob.add(inc_rec);
        off.term_ptr = blob.add(term_ptr);
        off.mem_var = blob.add(mem_var);
        off.mem_exp = blob.add(mem_exp);
        if (M->is_float) {
            std::vector<float> af(n_slots), tf(n_iterms);
            for (int32_t i = 0; i < n_slots; ++i) af[i] = (float)aconst_d[i];
            for (int32_t i = 0; i < n_iterms; ++i) tf[i] = (float)tcoef_d[i];
            off.aconst_f = blob.add(af); off.aconst_d = blob.add(aconst_d);
            off.tcoef_f = blob.add(tf); off.tcoef_d = blob.add(tcoef_d);
        } else {
            off.aconst_i = blob.add(aconst_i); off.tcoef_i = blob.add(tcoef_i);
        }
        dm.n_slots = n_slots;
        dm.n_iterms = n_iterms;
        M->cache_elems = n_slots;
    }
    dm.n_levels = M->n_levels;

    // ---- upload
    cudaError_t e = cudaMalloc(&M->dmem, blob.host.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(model)");
    M->dbytes = blob.host.size();
    e = cudaMemcpy(M->dmem, blob.host.data(), blob.host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(model)");
    void* b = M->dmem;
    dm.meta = at<VarMeta>(b, off.meta);
    dm.lvl_ptr = at<int32_t>(b, off.lvl_ptr);
    dm.lvl_vars = at<int32_t>(b, off.lvl_vars);
    dm.lvl_rec = at<sa::LevelRec>(b, off.lvl_rec);
    if (dm.kind == sa::KIND_QUIO) {
        dm.adj_col = at<int32_t>(b, off.adj_col);
        if (M->is_float) {
            dm.adj_f = at<float>(b, off.adj_f);
            dm.adj_d = off.adj_d == SIZE_MAX ? nullptr : at<double>(b, off.adj_d);
            dm.lin_f = at<float>(b, off.lin_f); dm.lin_d = at<double>(b, off.lin_d);
            dm.diag_f = at<float>(b, off.diag_f); dm.diag_d = at<double>(b, off.diag_d);
        } else {
            dm.adj_i = at<int64_t>(b, off.adj_i); dm.lin_i = at<int64_t>(b, off.lin_i);
            dm.diag_i = at<int64_t>(b, off.diag_i);
        }
    } else {
        dm.slot_base = at<int32_t>(b, off.slot_base);
        dm.omega = at<uint64_t>(b, off.omega);
        dm.inc_term = at<int32_t>(b, off.inc_term);
        dm.inc_exp = at<int32_t>(b, off.inc_exp);
        dm.inc_rec = at<int32_t>(b, off.inc_rec);
        dm.term_ptr = at<int32_t>(b, off.term_ptr);
        dm.mem_var = at<int32_t>(b, off.mem_var);
        dm.mem_exp = at<int32_t>(b, off.mem_exp);
        if (M->is_float) {
            dm.aconst_f = at<float>(b, off.aconst_f); dm.aconst_d = at<double>(b, off.aconst_d);
            dm.tcoef_f = at<float>(b, off.tcoef_f); dm.tcoef_d = at<double>(b, off.tcoef_d);
        } else {
            dm.aconst_i = at<int64_t>(b, off.aconst_i); dm.tcoef_i = at<int64_t>(b, off.tcoef_i);
        }
    }
    return SA_OK;
}


sa_status compile_model(sa_model* M, int32_t n, const int64_t* lower, const int64_t* upper, int64_t n_terms,
                        const int64_t* term_offsets, const int32_t* term_vars, const void* coeffs,
                        sa_coef_type ct) {
    M->n = n;
    M->is_float = (ct == SA_COEF_F32 || ct == SA_COEF_F64);
    M->f32_coeffs = (ct == SA_COEF_F32);
    std::vector<int32_t> lo(n);
    std::vector<uint32_t> width(n);
    for (int32_t k = 0; k < n; ++k) {
        if (lower[k] > upper[k]) return fail(SA_ERR_INVALID, "lower bound above upper bound at variable " + std::to_string(k));
        if (lower[k] < INT32_MIN || upper[k] > INT32_MAX)
            return fail(SA_ERR_UNSUPPORTED, "bounds must fit int32 (variable " + std::to_string(k) + ")");
        if (upper[k] - lower[k] > (int64_t)INT32_MAX)
            return fail(SA_ERR_INVALID, "range u-l must be below 2^31 (variable " + std::to_string(k) + ")");
        lo[k] = (int32_t)lower[k];
        width[k] = (uint32_t)(upper[k] - lower[k]);
        M->max_width = std::max(M->max_width, width[k]);
    }
    if (term_offsets == nullptr && n_terms > 0) return fail(SA_ERR_INVALID, "term_offsets is NULL");
    if (n_terms > 0 && term_offsets[0] != 0) return fail(SA_ERR_INVALID, "term_offsets[0] must be 0");
    for (int64_t t = 0; t < n_terms; ++t)
        if (term_offsets[t + 1] < term_offsets[t]) return fail(SA_ERR_INVALID, "term_offsets must be non-decreasing");
    const int64_t flat = n_terms > 0 ? term_offsets[n_terms] : 0;
    for (int64_t j = 0; j < flat; ++j)
        if (term_vars[j] < 0 || term_vars[j] >= n) return fail(SA_ERR_INVALID, "variable index out of range in term list");

    // ---- merge equal multisets (Sect. 2)
    std::unordered_map<std::string, size_t> index;
    std::vector<MergedTerm> terms;
    std::vector<Member> pool;
    __int128 const_i = 0;
    double const_d = 0.0;
    std::vector<int32_t> buf;
    for (int64_t t = 0; t < n_terms; ++t) {
        __int128 ci = 0;
        double cf = 0.0;
        switch (ct) {
        case SA_COEF_I32: ci = ((const int32_t*)coeffs)[t]; break;
        case SA_COEF_I64: ci = ((const int64_t*)coeffs)[t]; break;
        case SA_COEF_F32: cf = ((const float*)coeffs)[t]; break;
        case SA_COEF_F64: cf = ((const double*)coeffs)[t]; break;
        default: return fail(SA_ERR_INVALID, "unknown coefficient type");
        }
        if (M->is_float && !std::isfinite(cf)) return fail(SA_ERR_INVALID, "non-finite coefficient in term " + std::to_string(t));
        buf.assign(term_vars + term_offsets[t], term_vars + term_offsets[t + 1]);
        if (buf.empty()) {
            const_i += ci;
            const_d += cf;
            continue;
        }
        std::sort(buf.begin(), buf.end());
        std::string key(reinterpret_cast<const char*>(buf.data()), buf.size() * sizeof(int32_t));
        auto it = index.find(key);
        MergedTerm* cur;
        if (it == index.end()) {
            MergedTerm mt;
            mt.moff = (int64_t)pool.size();
            for (size_t i = 0; i < buf.size();) {
                size_t j = i;
                while (j < buf.size() && buf[j] == buf[i]) ++j;
                pool.push_back({buf[i], (int32_t)(j - i)});
                i = j;
            }
            mt.nmem = (int32_t)(pool.size() - mt.moff);
            mt.ci = ci;
            mt.cf = cf;
            index.emplace(std::move(key), terms.size());
            terms.push_back(std::move(mt));
            cur = &terms.back();
        } else {
            cur = &terms[it->second];
            cur->ci += ci;
            cur->cf += cf;
        }
        const __int128 lim = (__int128)1 << 100;
        if (!M->is_float && (cur->ci > lim || cur->ci < -lim)) return fail(SA_ERR_OVERFLOW, "merged coefficient overflows");
    }
    return compile_terms(M, n, lower, upper, lo, width, terms, pool, const_i, const_d);
}

// RAII holder of stream-ordered device temporaries
struct Temps {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Temps(cudaStream_t s) : st(s) {}
    cudaError_t alloc(void** p, size_t bytes) {
        cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~Temps() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

}  // namespace

extern "C" {

__attribute__((visibility("hidden"))) int sa_internal_model_view(const sa_model* M, sa::ModelView* v);

sa_status sa_model_create(sa_model** out, int32_t n_vars, const int64_t* lower, const int64_t* upper,
                          int64_t n_terms, const int64_t* term_offsets, const int32_t* term_vars, const void* coeffs,
                          sa_coef_type coef_type) {
    if (out == nullptr) return fail(SA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n_vars <= 0) return fail(SA_ERR_INVALID, "n_vars must be positive");
    if (lower == nullptr || upper == nullptr) return fail(SA_ERR_INVALID, "bounds are NULL");
    if (n_terms < 0) return fail(SA_ERR_INVALID, "n_terms is negative");
    if (n_terms > 0 && (term_vars == nullptr && term_offsets[n_terms] > 0)) return fail(SA_ERR_INVALID, "term_vars is NULL");
    if (n_terms > 0 && coeffs == nullptr) return fail(SA_ERR_INVALID, "coeffs is NULL");
    if ((int)coef_type < 0 || (int)coef_type > 3) return fail(SA_ERR_INVALID, "unknown coefficient type");
    sa_model* M = new sa_model();
    cudaGetDevice(&M->device);
    sa_status st = compile_model(M, n_vars, lower, upper, n_terms, term_offsets, term_vars, coeffs, coef_type);
    if (st != SA_OK) {
        if (M->dmem) cudaFree(M->dmem);
        delete M;
        return st;
    }
    *out = M;
    return SA_OK;
}

void sa_model_destroy(sa_model* model) {
    if (!model) return;
    if (model->dmem) cudaFree(model->dmem);
    delete model;
}

sa_status sa_model_create_quio_dense(sa_model** out, int32_t n, const int64_t* lower, const int64_t* upper,
                                     const void* h, const void* J, sa_coef_type coef_type) {
    if (out == nullptr) return fail(SA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n <= 0) return fail(SA_ERR_INVALID, "n_vars must be positive");
    if (!lower || !upper || !h || !J) return fail(SA_ERR_INVALID, "NULL argument");
    if ((int)coef_type < 0 || (int)coef_type > 3) return fail(SA_ERR_INVALID, "unknown coefficient type");
    sa_model* M = new sa_model();
    cudaGetDevice(&M->device);
    M->n = n;
    M->is_float = (coef_type == SA_COEF_F32 || coef_type == SA_COEF_F64);
    M->f32_coeffs = (coef_type == SA_COEF_F32);
    std::vector<int32_t> lo(n);
    std::vector<uint32_t> width(n);
    auto bad = [&](sa_status st, const std::string& msg) {
        delete M;
        return fail(st, msg);
    };
    for (int32_t k = 0; k < n; ++k) {
        if (lower[k] > upper[k]) return bad(SA_ERR_INVALID, "lower bound above upper bound at variable " + std::to_string(k));
        if (lower[k] < INT32_MIN || upper[k] > INT32_MAX) return bad(SA_ERR_UNSUPPORTED, "bounds must fit int32");
        if (upper[k] - lower[k] > (int64_t)INT32_MAX) return bad(SA_ERR_INVALID, "range u-l must be below 2^31");
        lo[k] = (int32_t)lower[k];
        width[k] = (uint32_t)(upper[k] - lower[k]);
        M->max_width = std::max(M->max_width, width[k]);
    }
    auto val = [&](const void* a, size_t i, __int128& ci, double& cf) {
        ci = 0;
        cf = 0.0;
        switch (coef_type) {
        case SA_COEF_I32: ci = ((const int32_t*)a)[i]; break;
        case SA_COEF_I64: ci = ((const int64_t*)a)[i]; break;
        case SA_COEF_F32: cf = ((const float*)a)[i]; break;
        default: cf = ((const double*)a)[i]; break;
        }
        return M->is_float ? (cf != 0.0) : (ci != 0);
    };
    std::vector<MergedTerm> terms;
    std::vector<Member> pool;
    __int128 ci;
    double cf;
    for (int32_t k = 0; k < n; ++k) {
        if (val(h, k, ci, cf)) {
            if (M->is_float && !std::isfinite(cf)) return bad(SA_ERR_INVALID, "non-finite coefficient");
            MergedTerm t;
            t.moff = (int64_t)pool.size();
            t.nmem = 1;
            t.ci = ci;
            t.cf = cf;
            pool.push_back({k, 1});
            terms.push_back(t);
        }
    }
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t j = i; j < n; ++j) {
            if (!val(J, (size_t)i * n + j, ci, cf)) continue;
            if (M->is_float && !std::isfinite(cf)) return bad(SA_ERR_INVALID, "non-finite coefficient");
            MergedTerm t;
            t.moff = (int64_t)pool.size();
            t.ci = ci;
            t.cf = cf;
            if (i == j) {
                pool.push_back({i, 2});
                t.nmem = 1;
            } else {
                pool.push_back({i, 1});
                pool.push_back({j, 1});
                t.nmem = 2;
            }
            terms.push_back(t);
        }
    }
    sa_status st = compile_terms(M, n, lower, upper, lo, width, terms, pool, 0, 0.0);
    if (st != SA_OK) {
        if (M->dmem) cudaFree(M->dmem);
        delete M;
        return st;
    }
    *out = M;
    return SA_OK;
}

sa_status sa_model_get_info(const sa_model* M, sa_model_info* info) {
    if (!M || !info) return fail(SA_ERR_INVALID, "NULL argument");
    info->n_vars = M->n;
    info->is_float = M->is_float;
    info->is_quadratic = M->quadratic;
    info->max_exponent = M->max_exp;
    info->max_order = M->max_order;
    info->all_multilinear = M->multilinear;
    info->n_terms = M->n_terms;
    info->n_links = M->n_links;
    info->n_levels = M->n_levels;
    info->max_width = (int32_t)M->max_width;
    info->device_bytes = (int64_t)M->dbytes;
    return SA_OK;
}

sa_status sa_default_temperatures(const sa_model* M, double* t_max, double* t_min) {
    if (!M || !t_max || !t_min) return fail(SA_ERR_INVALID, "NULL argument");
    *t_max = -M->de_max / std::log(0.5);
    *t_min = -M->de_min / std::log(0.001);
    return SA_OK;
}

sa_status sa_run(const sa_model* M, const sa_run_params* p, int32_t* out_states, void* out_energies,
                 uint64_t* out_accepts, void* stream) {
    if (!M || !p) return fail(SA_ERR_INVALID, "NULL model or params");
    if (!out_states || !out_energies) return fail(SA_ERR_INVALID, "NULL output");
    if (p->rule < 0 || p->rule > 2) return fail(SA_ERR_INVALID, "unknown rule");
    if (p->n_sweeps < 1 || p->n_replicas < 1) return fail(SA_ERR_INVALID, "n_sweeps and n_replicas must be positive");
    if (p->trace && (p->trace_replicas < 0 || p->trace_replicas > p->n_replicas))
        return fail(SA_ERR_INVALID, "trace_replicas out of range");
    if (p->rule == SA_OPT_METROPOLIS && M->max_exp > 4)
        return fail(SA_ERR_UNSUPPORTED, "optimal-transition Metropolis needs exponents <= 4");
    if ((p->best_states == nullptr) != (p->best_energies == nullptr))
        return fail(SA_ERR_INVALID, "best_states and best_energies are given together");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != M->device) return fail(SA_ERR_INVALID, "model belongs to another device");
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t S = p->n_sweeps, R = p->n_replicas, n = M->n;
    const bool want_best = p->best_states != nullptr;

    // ---- schedule (Sect. 3.1) and OTM ratio (Sect. 3.3.3)
    std::vector<float> tab(2 * (size_t)S);
    if (const char* err = sa::plan_schedule(M->de_max, M->de_min, S, p->t_max, p->t_min, p->temperatures, tab.data()))
        return fail(SA_ERR_INVALID, err);

    // ---- launch shape and per-replica state layout
    sa::ModelView view;
    sa_internal_model_view(M, &view);
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev);
    sa::RunPlan plan{};
    if (const char* err = sa::plan_run_shape(sa::plan_model(view), R, p->threads_per_replica, p->replicas_per_block,
                                             (p->flags & SA_FLAG_STATE_IN_GLOBAL) != 0, dev_sms,
                                             sa::sweep_max_shared_optin(), &plan))
        return fail(SA_ERR_INVALID, err);
    const bool in_global = plan.in_global != 0;
    const int rpc = plan.rpc, tpr = plan.tpr, blocks = plan.blocks;
    const size_t rep_bytes = (size_t)plan.rep_bytes, shared = (size_t)plan.shared_bytes;

    // ---- device temporaries and host/device outputs
    Temps tmp(st);
    cudaError_t e;
    const bool states_dev = is_device_ptr(out_states);
    const bool en_dev = is_device_ptr(out_energies);
    const bool acc_dev = out_accepts == nullptr || is_device_ptr(out_accepts);
    const bool bst_dev = !want_best || is_device_ptr(p->best_states);
    const bool ben_dev = !want_best || is_device_ptr(p->best_energies);
    const bool sync_needed = !states_dev || !en_dev || !acc_dev || !bst_dev || !ben_dev || p->report != nullptr;
    float* d_tab = nullptr;
    if ((e = tmp.alloc((void**)&d_tab, tab.size() * sizeof(float))) != cudaSuccess) return cuda_fail(e, "alloc schedule");
    if ((e = cudaMemcpyAsync(d_tab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "copy schedule");
    int32_t* d_states = out_states;
    void* d_en = out_energies;
    unsigned long long* d_acc = (unsigned long long*)out_accepts;
    if (!states_dev && (e = tmp.alloc((void**)&d_states, (size_t)R * n * 4)) != cudaSuccess) return cuda_fail(e, "alloc states");
    if (!en_dev && (e = tmp.alloc(&d_en, (size_t)R * 8)) != cudaSuccess) return cuda_fail(e, "alloc energies");
    if (!acc_dev && (e = tmp.alloc((void**)&d_acc, (size_t)R * 8)) != cudaSuccess) return cuda_fail(e, "alloc accepts");
    int32_t* d_bst = p->best_states;
    void* d_ben = p->best_energies;
    if (!bst_dev && (e = tmp.alloc((void**)&d_bst, (size_t)R * n * 4)) != cudaSuccess) return cuda_fail(e, "alloc best states");
    if (!ben_dev && (e = tmp.alloc(&d_ben, (size_t)R * 8)) != cudaSuccess) return cuda_fail(e, "alloc best energies");
    const int32_t* d_init = p->init_states;
    if (p->init_states && !is_device_ptr(p->init_states)) {
        int32_t* di = nullptr;
        if ((e = tmp.alloc((void**)&di, (size_t)R * n * 4)) != cudaSuccess) return cuda_fail(e, "alloc init");
        if ((e = cudaMemcpyAsync(di, p->init_states, (size_t)R * n * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "copy init");
        d_init = di;
    }
    uint8_t* gstate = nullptr;
    if (in_global && (e = tmp.alloc((void**)&gstate, (size_t)R * rep_bytes)) != cudaSuccess) return cuda_fail(e, "alloc state");
    unsigned int* d_drift = nullptr;
    if (p->report && M->is_float) {
        if ((e = tmp.alloc((void**)&d_drift, 16)) != cudaSuccess) return cuda_fail(e, "alloc drift");
        cudaMemsetAsync(d_drift, 0, 16, st);
    }

    sa::SweepArgs a{};
    a.m = M->dm;
    a.R = R;
    a.S = S;
    a.key0 = (uint32_t)(p->seed & 0xFFFFFFFFull);
    a.key1 = (uint32_t)(p->seed >> 32);
    a.inst = p->instance_id;
    a.refresh_interval = p->refresh_interval > 0 ? p->refresh_interval : 50;
    a.speculate = (p->flags & SA_FLAG_NO_SPECULATION) ? 0 : 1;
    a.beta = d_tab;
    a.ratio = d_tab + S;
    a.init_states = d_init;
    a.out_states = d_states;
    a.out_energies = d_en;
    a.out_accepts = d_acc;
    a.trace = p->trace;
    a.trace_R = p->trace ? p->trace_replicas : 0;
    a.energy_trace = p->energy_trace;
    a.best_states = d_bst;
    a.best_energies = d_ben;
    a.drift_bits = d_drift;
    a.gstate = gstate;
    sa::plan_apply(plan, a);

    // ---- time slicing: when the replicas need more than one wave of resident
    // thread groups and the last wave would leave slots idle, one cooperative
    // launch lets the resident groups claim (replica, chunk of sweeps) tasks
    // (sa::slice_chunk_sweeps); results are those of the plain launch
    int grid_sliced = 0;
    unsigned int* d_status = nullptr;
    if (!in_global && !(p->flags & SA_FLAG_NO_TIME_SLICING) && shared + 64 <= (size_t)sa::sweep_max_shared_optin()) {
        int bps = 0;
        if (sa::launch_sweep_sliced(a, M->zbytes, p->rule, 0, rpc * tpr, shared, stream, &bps) == 0 && bps > 0) {
            const int64_t slots = (int64_t)dev_sms * bps * rpc;
            const int64_t waves = (R + slots - 1) / slots;
            if (R > slots && (double)R < 0.95 * (double)(waves * slots)) grid_sliced = dev_sms * bps;
        } else {
            cudaGetLastError();
        }
    }
    if (grid_sliced > 0) {
        a.handoff_bytes = (int64_t)align_up((size_t)plan.off_ctl + (size_t)tpr * 24, 16);
        uint8_t* d_hand = nullptr;
        if ((e = tmp.alloc((void**)&d_hand, (size_t)R * (size_t)a.handoff_bytes + (size_t)R * 4 + 16)) !=
            cudaSuccess)
            return cuda_fail(e, "alloc handoff");
        a.handoff = d_hand;
        a.handoff_flag = reinterpret_cast<unsigned int*>(d_hand + (size_t)R * (size_t)a.handoff_bytes);
        d_status = a.handoff_flag + R;
        a.status = d_status;
        cudaMemsetAsync(a.handoff_flag, 0, (size_t)R * 4 + 16, st);
    }

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (p->report) {
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
        cudaEventRecord(ev0, st);
    }
    int le = 1;
    if (grid_sliced > 0) {
        le = sa::launch_sweep_sliced(a, M->zbytes, p->rule, grid_sliced, rpc * tpr, shared, stream, nullptr);
        if (le != 0) {
            cudaGetLastError();   // the cooperative launch was refused: run the plain launch instead
            grid_sliced = 0;
            d_status = nullptr;
        }
    }
    if (grid_sliced == 0) le = sa::launch_sweep(a, M->zbytes, p->rule, !in_global, blocks, rpc * tpr, shared, stream);
    if (le != 0) return cuda_fail((cudaError_t)le, "sweep launch");
    if (p->report) cudaEventRecord(ev1, st);
    if (want_best && M->is_float) {
        // the chosen states' energies in FP64 (the kernel chose by the tracked energy)
        int32_t* d_bad = nullptr;
        if ((e = tmp.alloc((void**)&d_bad, 16)) != cudaSuccess) return cuda_fail(e, "alloc flag");
        cudaMemsetAsync(d_bad, 0, 16, st);
        sa::EnergyArgs ea{M->dm, d_bst, R, d_ben, d_bad};
        if ((le = sa::launch_energy(ea, stream)) != 0) return cuda_fail((cudaError_t)le, "energy launch");
    }
    if (!bst_dev && (e = cudaMemcpyAsync(p->best_states, d_bst, (size_t)R * n * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "copy best states");
    if (!ben_dev && (e = cudaMemcpyAsync(p->best_energies, d_ben, (size_t)R * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "copy best energies");

    if (!states_dev && (e = cudaMemcpyAsync(out_states, d_states, (size_t)R * n * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "copy states");
    if (!en_dev && (e = cudaMemcpyAsync(out_energies, d_en, (size_t)R * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "copy energies");
    if (!acc_dev && (e = cudaMemcpyAsync(out_accepts, d_acc, (size_t)R * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "copy accepts");
    unsigned int drift_h = 0;
    if (d_drift && (e = cudaMemcpyAsync(&drift_h, d_drift, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "copy drift");
    unsigned int status_h = 0;
    if (d_status && sync_needed &&
        (e = cudaMemcpyAsync(&status_h, d_status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "copy status");
    if (sync_needed) {
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sa_run");
        if (status_h) return fail(SA_ERR_TIMEOUT, "a state handoff between thread groups timed out");
    }
    if (p->report) {
        sa_run_report* rp = p->report;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        float dr;
        std::memcpy(&dr, &drift_h, 4);
        rp->max_refresh_drift = M->is_float ? (double)dr : 0.0;
        rp->replicas_per_block = rpc;
        rp->threads_per_replica = tpr;
        rp->state_in_global = in_global ? 1 : 0;
        rp->shared_bytes = (int32_t)shared;
        rp->blocks = grid_sliced > 0 ? grid_sliced : blocks;
        rp->n_levels = M->n_levels;
        rp->kernel_ms = ms;
        rp->time_sliced = grid_sliced > 0 ? 1 : 0;
    }
    return SA_OK;
}

sa_status sa_energy(const sa_model* M, const int32_t* states, int64_t n_states, void* energies, void* stream) {
    if (!M) return fail(SA_ERR_INVALID, "NULL model");
    if (n_states < 0) return fail(SA_ERR_INVALID, "n_states is negative");
    if (n_states == 0) return SA_OK;
    if (!states || !energies) return fail(SA_ERR_INVALID, "NULL buffer");
    cudaStream_t st = (cudaStream_t)stream;
    Temps tmp(st);
    cudaError_t e;
    const size_t sbytes = (size_t)n_states * M->n * 4;
    const int32_t* d_states = states;
    if (!is_device_ptr(states)) {
        int32_t* ds = nullptr;
        if ((e = tmp.alloc((void**)&ds, sbytes)) != cudaSuccess) return cuda_fail(e, "alloc states");
        if ((e = cudaMemcpyAsync(ds, states, sbytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(e, "copy states");
        d_states = ds;
    }
    const bool en_dev = is_device_ptr(energies);
    void* d_en = energies;
    if (!en_dev && (e = tmp.alloc(&d_en, (size_t)n_states * 8)) != cudaSuccess) return cuda_fail(e, "alloc energies");
    int32_t* d_bad = nullptr;
    if ((e = tmp.alloc((void**)&d_bad, 16)) != cudaSuccess) return cuda_fail(e, "alloc flag");
    cudaMemsetAsync(d_bad, 0, 16, st);
    sa::EnergyArgs a{M->dm, d_states, n_states, d_en, d_bad};
    int le = sa::launch_energy(a, stream);
    if (le != 0) return cuda_fail((cudaError_t)le, "energy launch");
    int bad = 0;
    if ((e = cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(e, "copy flag");
    if (!en_dev && (e = cudaMemcpyAsync(energies, d_en, (size_t)n_states * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(e, "copy energies");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "sa_energy");
    if (bad) return fail(SA_ERR_INVALID, "a state value lies outside its bounds");
    return SA_OK;
}

const char* sa_last_error(void) { return g_last_error.c_str(); }

// Internal view of a compiled model for other translation units of this library.
__attribute__((visibility("hidden"))) int sa_internal_model_view(const sa_model* M, sa::ModelView* v) {
    if (!M || !v) return 0;
    v->dm = M->dm;
    v->device = M->device;
    v->n = M->n;
    v->is_float = M->is_float ? 1 : 0;
    v->max_exp = M->max_exp;
    v->zbytes = M->zbytes;
    v->cache_elems = M->cache_elems;
    v->n_levels = M->n_levels;
    v->max_link_len = M->max_link_len;
    v->de_max = M->de_max;
    v->de_min = M->de_min;
    return 1;
}

// Device bytes held by a model.
__attribute__((visibility("hidden"))) int64_t sa_internal_model_bytes(const sa_model* M) { return M ? (int64_t)M->dbytes : 0; }

// Records a failure message for sa_last_error() from another translation unit.
__attribute__((visibility("hidden"))) void sa_internal_set_error(const char* msg) { g_last_error = msg ? msg : ""; }

const char* sa_version(void) { return "paper_2511_17245_gb300 0.1 (sm_103a)"; }

}  // extern "C"
