// sweep.cuh -- the single-variable update sweep of direct SA (arXiv:2511.17245,
// Sect. 3) for sm_103a.
//
// Layout and parallel structure
//   * One group of `tpr` threads (whole warps) owns one replica (an
//     independent SA run).  A block holds `rpc` such groups; each group
//     synchronises on its own named barrier (id 1 + slot).
//   * A replica's state -- the offsets z_k - l_k (1, 2 or 4 bytes) and the
//     cached coefficients (QUIO: f_k = J_k + sum_{i != k} J_ik z_i, the
//     paper's c^(1)_k minus 2 J_kk z_k; HUIO: a_k^(m) of Eq. energy_diff_poly)
//     -- lives in shared memory when it fits, else in a global slab.
//   * Sequential visit order (Sect. 3.1) is kept exactly: the host splits the
//     index sequence 0..N-1 into dependency levels (level(k) = 1 + max level
//     of the neighbours j < k that share a term with k).  Variables of one
//     level share no term, so their decisions read disjoint state and their
//     cache updates commute; the group runs a level in parallel and
//     barriers between levels.  For integer models this reproduces the
//     sequential trajectory bit for bit.
//   * Per attempt: one Philox4x32-10 block with counter (k, s, r, instance).
//
// Decision arithmetic (shared convention with the CPU oracle):
//   Metropolis / OTM acceptance: dE <= 0, or U(x1) < expf(-fp32(dE) * beta_s).
//   Heat bath: weights expf(-fp32(dE_v - dE_min) * beta_s), compensated fp32
//   sums, smallest v with C_v >= Uc(x0) * C_total; multilinear variables use
//   the inverse transform of Eq. inverse_prob.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sa_internal.h"

namespace sa {
namespace dev {

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).
struct Words4 {
    uint32_t x0, x1, x2, x3;
};

__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ float unit_open_right(uint32_t x) { return __uint2float_rn(x >> 8) * 0x1p-24f; }
__device__ __forceinline__ float unit_open_left(uint32_t x) { return __uint2float_rn((x >> 8) + 1u) * 0x1p-24f; }
__device__ __forceinline__ uint32_t pick_below(uint32_t x, uint32_t m) { return __umulhi(x, m); }

// ------------------------------------------------------------------ numeric traits
template <class F>
struct Num;
template <>
struct Num<long long> {
    using Acc = long long;                 // energy accumulator
    static constexpr bool is_float = false;
    // int64 -> fp32, round to nearest.  On sm_103a the 64-bit conversion runs on
    // the FP64 pipe; values that fit int32 take the 32-bit conversion, which
    // rounds identically.
    __device__ static float to_f(long long v) {
        return (v == (long long)(int)v) ? __int2float_rn((int)v) : __ll2float_rn(v);
    }
};
template <>
struct Num<float> {
    using Acc = double;
    static constexpr bool is_float = true;
    __device__ static float to_f(float v) { return v; }
};

__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void atomic_add_field(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_field(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

// Floor division for int64 with positive divisor.
__device__ __forceinline__ long long floor_div(long long a, long long b) {
    long long q = a / b;
    if ((a % b != 0) && (a < 0)) --q;
    return q;
}

// ------------------------------------------------------------------ model accessors
template <class F>
struct Coef;
template <>
struct Coef<long long> {
    __device__ static long long adj(const DevModel& m, int i) { return m.adj_i[i]; }
    __device__ static long long lin(const DevModel& m, int k) { return m.lin_i[k]; }
    __device__ static long long diag(const DevModel& m, int k) { return m.diag_i[k]; }
    __device__ static long long aconst(const DevModel& m, int s) { return m.aconst_i[s]; }
    __device__ static long long tcoef(const DevModel& m, int t) { return m.tcoef_i[t]; }
};
template <>
struct Coef<float> {
    __device__ static float adj(const DevModel& m, int i) { return __ldg(m.adj_f + i); }
    __device__ static float lin(const DevModel& m, int k) { return __ldg(m.lin_f + k); }
    __device__ static float diag(const DevModel& m, int k) { return __ldg(m.diag_f + k); }
    __device__ static float aconst(const DevModel& m, int s) { return __ldg(m.aconst_f + s); }
    __device__ static float tcoef(const DevModel& m, int t) { return __ldg(m.tcoef_f + t); }
};

// Integer power by repeated multiplication (exponents are small).
template <class T>
__device__ __forceinline__ T ipow(T x, int e) {
    T r = T(1);
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

// ------------------------------------------------------------------ energy change
// QUIO (Eq. energy_diff_quad): dE(v) = (v - z) * (f + J_kk (v + z)), f = c1 - 2 J_kk z.
template <class F>
__device__ __forceinline__ F quio_delta(F f, F d, long long z, long long v) {
    if constexpr (Num<F>::is_float) {
        const float vf = __int2float_rn((int)v), zf = __int2float_rn((int)z);
        return (vf - zf) * fmaf(d, vf + zf, f);
    } else {
        return (v - z) * (f + d * (v + z));
    }
}

// HUIO (Eq. energy_diff_poly): dE(v) = sum_{m in Omega_k} a^(m) (v^m - z^m).
template <class F>
__device__ __forceinline__ F huio_delta(const F* a_slots, uint64_t omega, long long z, long long v) {
    F acc = F(0);
    if constexpr (Num<F>::is_float) {
        float pv = 1.f, pz = 1.f;
        const float vf = __int2float_rn((int)v), zf = __int2float_rn((int)z);
        int slot = 0;
        uint64_t msk = omega >> 1;
        while (msk) {
            pv *= vf;
            pz *= zf;
            if (msk & 1ull) acc = fmaf(a_slots[slot++], pv - pz, acc);
            msk >>= 1;
        }
    } else {
        long long pv = 1, pz = 1;
        int slot = 0;
        uint64_t msk = omega >> 1;
        while (msk) {
            pv *= v;
            pz *= z;
            if (msk & 1ull) acc += a_slots[slot++] * (pv - pz);
            msk >>= 1;
        }
    }
    return acc;
}

template <class F>
__device__ __forceinline__ bool le_zero(F x) { return x <= F(0); }

// Metropolis acceptance of Sect. 3.3.1 in the shared fp32 convention.
template <class F>
__device__ __forceinline__ bool metropolis_accept(F de, uint32_t xu, float beta) {
    if (de <= F(0)) return true;
    const float x = Num<F>::to_f(de) * beta;
    const float p = expf(-x);
    return unit_open_right(xu) < p;
}

// ------------------------------------------------------------------ per-variable view
// Everything the decision of variable k needs, for either model kind.
template <class F, int KIND>
struct VarView;

template <class F>
struct VarView<F, KIND_QUIO> {
    F f, d;
    __device__ F delta(long long z, long long v) const { return quio_delta<F>(f, d, z, v); }
    // float models: candidate and current value already as floats
    __device__ float delta_ff(float zf, float vf) const { return (vf - zf) * fmaf((float)d, vf + zf, (float)f); }
    __device__ bool linear() const { return d == F(0); }
    __device__ F lin_coef() const { return f; }
    __device__ int max_exp() const { return d == F(0) ? 1 : 2; }
    __device__ F coef(int m) const { return m == 1 ? f : (m == 2 ? d : F(0)); }
};

template <class F>
struct VarView<F, KIND_HUIO> {
    const F* a;
    uint64_t omega;
    __device__ F delta(long long z, long long v) const { return huio_delta<F>(a, omega, z, v); }
    __device__ float delta_ff(float zf, float vf) const {
        float acc = 0.f, pv = 1.f, pz = 1.f;
        int slot = 0;
        uint64_t msk = omega >> 1;
        while (msk) {
            pv *= vf;
            pz *= zf;
            if (msk & 1ull) acc = fmaf((float)a[slot++], pv - pz, acc);
            msk >>= 1;
        }
        return acc;
    }
    __device__ bool linear() const { return (omega & ~2ull) == 0; }
    __device__ F lin_coef() const { return (omega & 2ull) ? a[0] : F(0); }
    __device__ int max_exp() const { return omega ? 63 - __clzll(omega) : 0; }
    // coefficient of z^m (0 if absent)
    __device__ F coef(int m) const {
        if (!((omega >> m) & 1ull)) return F(0);
        const uint64_t below = omega & ((1ull << m) - 1ull);
        return a[__popcll(below >> 1)];
    }
};

// ------------------------------------------------------------------ OTM argmin
// argmin over v in [lo, lo+width], v != z, of dE(v); ties to the smallest v.
// Candidate set: lo, hi, z-1, z+1 and the integers around every local minimum
// of the continuous polynomial (exact for degree <= 2; for degree 3 and 4 the
// critical points are bracketed on the monotone pieces of P' and a window of
// integers around each is evaluated exactly).
template <class F, int KIND>
struct ArgminState {
    long long best_v;
    F best;
    bool have;
    __device__ void offer(const VarView<F, KIND>& vv, long long z, long long lo, long long hi, long long v) {
        if (v < lo || v > hi || v == z) return;
        const F de = vv.delta(z, v);
        if (!have || de < best || (de == best && v < best_v)) {
            best = de;
            best_v = v;
            have = true;
        }
    }
};

template <class F, int KIND>
__device__ long long opt_argmin(const VarView<F, KIND>& vv, long long z, long long lo, long long hi) {
    ArgminState<F, KIND> st{0, F(0), false};
    st.offer(vv, z, lo, hi, lo);
    st.offer(vv, z, lo, hi, hi);
    st.offer(vv, z, lo, hi, z - 1);
    st.offer(vv, z, lo, hi, z + 1);
    const int me = vv.max_exp();
    if (me == 2) {
        const F a1 = vv.coef(1), a2 = vv.coef(2);
        if (a2 > F(0)) {
            long long q;
            if constexpr (Num<F>::is_float) {
                // bounds fit int32 (model compiler), so the clamp and the
                // conversion back stay in 32-bit conversions (64-bit ones run on
                // the FP64 pipe); hi + 1 = 2^31 is the one value beyond int32
                float qv = floorf(-a1 / (2.f * a2));
                qv = fminf(fmaxf(qv, __int2float_rn((int)lo) - 1.f), __int2float_rn((int)hi) + 1.f);
                q = qv >= 2147483648.f ? 2147483648LL : (long long)__float2int_rz(qv);
            } else {
                q = floor_div(-a1, 2 * a2);
            }
            st.offer(vv, z, lo, hi, q);
            st.offer(vv, z, lo, hi, q + 1);
        }
    } else if (me >= 3) {
        // P'(x) = c0 + c1 x + c2 x^2 + c3 x^3 in double; pieces between the
        // roots of P'' are monotone; bisect each sign change on the integers.
        const double c0 = (double)vv.coef(1), c1 = 2.0 * (double)vv.coef(2);
        const double c2 = 3.0 * (double)vv.coef(3), c3 = 4.0 * (double)vv.coef(4);
        auto dp = [&](double x) { return ((c3 * x + c2) * x + c1) * x + c0; };
        double brk[4];
        int nb = 0;
        brk[nb++] = (double)lo;
        // roots of P''(x) = c1 + 2 c2 x + 3 c3 x^2
        const double qa = 3.0 * c3, qb = 2.0 * c2, qc = c1;
        if (qa != 0.0) {
            const double disc = qb * qb - 4.0 * qa * qc;
            if (disc > 0.0) {
                const double sq = sqrt(disc);
                const double t = -0.5 * (qb + (qb >= 0 ? sq : -sq));
                double r1 = t / qa, r2 = (t != 0.0) ? qc / t : r1;
                if (r1 > r2) { const double tmp = r1; r1 = r2; r2 = tmp; }
                if (r1 > (double)lo && r1 < (double)hi) brk[nb++] = r1;
                if (r2 > (double)lo && r2 < (double)hi && r2 != r1) brk[nb++] = r2;
            }
        } else if (qb != 0.0) {
            const double r = -qc / qb;
            if (r > (double)lo && r < (double)hi) brk[nb++] = r;
        }
        brk[nb++] = (double)hi;
        for (int p = 0; p + 1 < nb; ++p) {
            long long a = (long long)floor(brk[p]), b = (long long)ceil(brk[p + 1]);
            if (a < lo) a = lo;
            if (b > hi) b = hi;
            // window around each break point
            for (long long w = -2; w <= 2; ++w) st.offer(vv, z, lo, hi, a + w);
            const double fa = dp((double)a), fb = dp((double)b);
            if (fa < 0.0 && fb > 0.0) {          // P' increases through zero: local minimum
                long long L = a, H = b;          // dp(L) < 0 <= dp(H)
                while (H - L > 1) {
                    const long long mid = L + (H - L) / 2;
                    if (dp((double)mid) < 0.0) L = mid; else H = mid;
                }
                for (long long w = -2; w <= 3; ++w) st.offer(vv, z, lo, hi, L + w);
            }
        }
    }
    return st.have ? st.best_v : z;
}

// ------------------------------------------------------------------ heat bath
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Weights below exp(-(20 + ln n)) times the largest one are left out of the
// heat-bath sum: with n candidates their total is below e^-20 of the total,
// far inside the near-threshold margin of the decision.  Candidates are
// dropped only in whole blocks, and only when a lower bound of dE over the
// block proves every weight in it small.
__device__ __forceinline__ float hb_cut(uint32_t width) { return 20.f + logf((float)width + 1.f); }

// Lower bound of dE over the candidate values [v0, v1] of a QUIO variable:
// dE(v) = (v - z)(f + d (v + z)) is convex (d > 0) or concave (d <= 0) in v, so
// the minimum over an interval is at an endpoint or next to the vertex
// v* = -f / (2 d).
template <class F>
__device__ __forceinline__ F quio_interval_min(const VarView<F, KIND_QUIO>& vv, long long z, long long v0,
                                               long long v1) {
    F mnb = vv.delta(z, v0);
    const F e1 = vv.delta(z, v1);
    mnb = e1 < mnb ? e1 : mnb;
    if (vv.d > F(0)) {
        long long q;
        if constexpr (Num<F>::is_float) {
            float qv = floorf(-(float)vv.f / (2.f * (float)vv.d));
            qv = fminf(fmaxf(qv, (float)v0), (float)v1);
            q = (long long)qv;
        } else {
            q = floor_div(-vv.f, 2 * vv.d);
        }
        if (q >= v0 && q <= v1) { const F e = vv.delta(z, q); mnb = e < mnb ? e : mnb; }
        if (q + 1 >= v0 && q + 1 <= v1) { const F e = vv.delta(z, q + 1); mnb = e < mnb ? e : mnb; }
    }
    return mnb;
}

// Kept window [wb0, wb1] of the blocks of 32 values of a QUIO variable
// (blocks counted from lo; nblk = width / 32 + 1 on entry as wb1 + 1): for a
// convex variable (J_kk > 0) the block lower bound of dE falls and then rises,
// so the first and last kept blocks are found by bisection on either side of
// the vertex; otherwise (or if rounding hides the vertex block) every block.
template <class F>
__device__ __forceinline__ void hb_quio_window(const VarView<F, KIND_QUIO>& vv, long long z, long long lo,
                                               uint32_t width, F mn, float beta, uint32_t& wb0, uint32_t& wb1) {
    constexpr uint32_t B = 32;
    if (!(vv.d > F(0))) return;
    const uint32_t nblk = wb1 + 1;
    const float cutv = hb_cut(width);
    auto kept = [&](uint32_t b) -> bool {
        const long long v0 = lo + (long long)(b * B);
        const long long v1 = lo + (long long)min(width, b * B + (B - 1));
        return Num<F>::to_f(quio_interval_min<F>(vv, z, v0, v1) - mn) * beta <= cutv;
    };
    // block holding the minimum
    long long vstar;
    if constexpr (Num<F>::is_float) {
        float qv = floorf(-(float)vv.f / (2.f * (float)vv.d));
        qv = fminf(fmaxf(qv, (float)lo), (float)(lo + (long long)width));
        vstar = (long long)qv;
    } else {
        vstar = floor_div(-vv.f, 2 * vv.d);
        if (vstar < lo) vstar = lo;
        if (vstar > lo + (long long)width) vstar = lo + (long long)width;
    }
    const uint32_t bm = (uint32_t)(vstar - lo) / B;
    if (!kept(bm)) return;  // rounding: keep every block
    uint32_t a = 0, c = bm;  // first kept block in [0, bm]
    while (a < c) { const uint32_t mid = (a + c) / 2; if (kept(mid)) c = mid; else a = mid + 1; }
    wb0 = a;
    a = bm; c = nblk - 1;    // last kept block in [bm, nblk-1]
    while (a < c) { const uint32_t mid = (a + c + 1) / 2; if (kept(mid)) a = mid; else c = mid - 1; }
    wb1 = a;
}

// Explicit inverse CDF over all u-l+1 values (Eq. prob_heatbath).
// Integer models: three passes over the candidates (minimum dE, compensated
// total, compensated search) with fp32 weights expf(-fp32(dE_v - dE_min) beta),
// the convention shared with the oracle.
// Float models: the same three passes with the candidate value carried as an
// exact float counter (no integer conversions in the loop) and weights
// 2^((dE_min - dE_v) beta log2 e).
// QUIO variables skip blocks of 32 values whose weights are all negligible
// (see hb_cut); the minimum then comes from the interval bounds as well.
template <class F, int KIND>
__device__ long long heat_bath_general(const VarView<F, KIND>& vv, long long z, long long lo, uint32_t width,
                                       uint32_t xu, float beta) {
    constexpr uint32_t B = 32;
    const uint32_t nblk = width / B + 1;
    // minimum over all values (current value included: dE = 0)
    F mn = F(0);
    if constexpr (KIND == KIND_QUIO) {
        const F e = quio_interval_min<F>(vv, z, lo, lo + (long long)width);
        mn = e < mn ? e : mn;
    } else {
        for (uint32_t i = 0; i <= width; ++i) {
            const F de = vv.delta(z, lo + (long long)i);
            mn = de < mn ? de : mn;
        }
    }
    // kept window [wb0, wb1] of blocks
    uint32_t wb0 = 0, wb1 = nblk - 1;
    if constexpr (KIND == KIND_QUIO) hb_quio_window<F>(vv, z, lo, width, mn, beta, wb0, wb1);
    if constexpr (Num<F>::is_float) {
        const float zf = __int2float_rn((int)z), v0f = __int2float_rn((int)lo);
        const float b2 = beta * 1.4426950408889634f, mb = (float)mn * b2;
        float sum = 0.f, comp = 0.f;
        for (uint32_t b = wb0; b <= wb1; ++b) {
            const uint32_t e = min(width, b * B + (B - 1));
            float vf = v0f + (float)(b * B);
            for (uint32_t i = b * B; i <= e; ++i, vf += 1.f) {
                const float w = ex2_ftz(fmaf(-vv.delta_ff(zf, vf), b2, mb));
                const float y = w - comp;
                const float t = sum + y;
                comp = (t - sum) - y;
                sum = t;
            }
        }
        const float thr = unit_open_left(xu) * sum;
        float run = 0.f, c2 = 0.f;
        long long last = lo;
        for (uint32_t b = wb0; b <= wb1; ++b) {
            const uint32_t e = min(width, b * B + (B - 1));
            float vf = v0f + (float)(b * B);
            for (uint32_t i = b * B; i <= e; ++i, vf += 1.f) {
                const float w = ex2_ftz(fmaf(-vv.delta_ff(zf, vf), b2, mb));
                const float y = w - c2;
                const float t = run + y;
                c2 = (t - run) - y;
                run = t;
                last = lo + (long long)i;
                if (run >= thr) return last;
            }
        }
        return last;
    } else {
        float sum = 0.f, comp = 0.f;
        for (uint32_t b = wb0; b <= wb1; ++b) {
            const uint32_t e = min(width, b * B + (B - 1));
            for (uint32_t i = b * B; i <= e; ++i) {
                const F de = vv.delta(z, lo + (long long)i);
                const float w = expf(-(Num<F>::to_f(de - mn) * beta));
                const float y = w - comp;
                const float t = sum + y;
                comp = (t - sum) - y;
                sum = t;
            }
        }
        const float thr = unit_open_left(xu) * sum;
        float run = 0.f, c2 = 0.f;
        long long last = lo;
        for (uint32_t b = wb0; b <= wb1; ++b) {
            const uint32_t e = min(width, b * B + (B - 1));
            for (uint32_t i = b * B; i <= e; ++i) {
                const F de = vv.delta(z, lo + (long long)i);
                const float w = expf(-(Num<F>::to_f(de - mn) * beta));
                const float y = w - c2;
                const float t = run + y;
                c2 = (t - run) - y;
                run = t;
                last = lo + (long long)i;
                if (run >= thr) return last;
            }
        }
        return last;
    }
}

// ------------------------------------------------------------------ warp-parallel heat bath
// A pair hi + lo added with Knuth's TwoSum: the rounding error of hi + hi' is
// kept in lo, so that sums over many lanes stay within a few ulp.
struct CompF {
    float hi, lo;
};
__device__ __forceinline__ CompF comp_add(CompF a, CompF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return {s, e + (a.lo + b.lo)};
}

template <class T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// The inverse CDF of Eq. prob_heatbath for one variable, evaluated by the 32
// lanes of a warp together (all lanes call it with the same arguments and
// receive the same value).  Same weights, candidate window and pick rule as
// heat_bath_general (smallest v with C_v >= Uc C_total):
//   1. dE_min: closed form for QUIO, lane-strided minimum for HUIO;
//   2. the kept candidates [c0, c1] are cut into 32 contiguous segments, one
//      per lane; each lane sums its weights (Kahan) and the warp forms the
//      inclusive prefix of the segment sums with compensated pairs;
//   3. the first lane whose inclusive prefix reaches Uc C_total walks its
//      segment from its exclusive prefix and picks the value.
// The lanes therefore touch each candidate once for the total and one
// segment once more for the pick, instead of one lane walking all of them.
template <class F, int KIND>
__device__ long long heat_bath_warp(const VarView<F, KIND>& vv, long long z, long long lo, uint32_t width,
                                    uint32_t xu, float beta, int lane) {
    constexpr uint32_t B = 32;
    constexpr unsigned full = 0xffffffffu;
    F mn = F(0);
    if constexpr (KIND == KIND_QUIO) {
        const F e = quio_interval_min<F>(vv, z, lo, lo + (long long)width);
        mn = e < mn ? e : mn;
    } else {
        for (uint32_t i = (uint32_t)lane; i <= width; i += 32) {
            const F de = vv.delta(z, lo + (long long)i);
            mn = de < mn ? de : mn;
        }
        mn = warp_min(mn);
    }
    uint32_t wb0 = 0, wb1 = width / B;
    if constexpr (KIND == KIND_QUIO) hb_quio_window<F>(vv, z, lo, width, mn, beta, wb0, wb1);
    const uint32_t c0 = wb0 * B, c1 = min(width, wb1 * B + (B - 1));
    const uint32_t m = (c1 - c0) / 32 + 1;                 // segment length
    const uint32_t s0 = c0 + (uint32_t)lane * m;           // this lane's segment [s0, s1]
    const bool has = s0 <= c1;
    const uint32_t s1 = has ? min(c1, s0 + (m - 1)) : 0u;
    const float zf = __int2float_rn((int)z), v0f = __int2float_rn((int)lo);
    const float b2 = beta * 1.4426950408889634f, mb = Num<F>::to_f(mn) * b2;
    auto weight = [&](uint32_t i) -> float {
        if constexpr (Num<F>::is_float) {
            return ex2_ftz(fmaf(-vv.delta_ff(zf, v0f + (float)i), b2, mb));
        } else {
            return expf(-(Num<F>::to_f(vv.delta(z, lo + (long long)i) - mn) * beta));
        }
    };
    float sum = 0.f, comp = 0.f;
    if (has) {
        for (uint32_t i = s0; i <= s1; ++i) {
            const float y = weight(i) - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
    }
    CompF v{sum, -comp};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const CompF u{__shfl_up_sync(full, v.hi, o), __shfl_up_sync(full, v.lo, o)};
        if (lane >= o) v = comp_add(u, v);
    }
    const float tot = __shfl_sync(full, v.hi, 31) + __shfl_sync(full, v.lo, 31);
    const float thr = unit_open_left(xu) * tot;
    CompF ex{__shfl_up_sync(full, v.hi, 1), __shfl_up_sync(full, v.lo, 1)};
    if (lane == 0) ex = CompF{0.f, 0.f};
    const unsigned hit = __ballot_sync(full, has && (v.hi + v.lo) >= thr);
    const unsigned nonempty = __ballot_sync(full, has);
    // rounding can leave the threshold above the last prefix: take the last segment
    const int sel = hit ? __ffs(hit) - 1 : 31 - __clz(nonempty);
    long long pick = 0;
    if (lane == sel) {
        pick = lo + (long long)s1;
        CompF run = ex;
        for (uint32_t i = s0; i <= s1; ++i) {
            run = comp_add(run, CompF{weight(i), 0.f});
            if (run.hi + run.lo >= thr) {
                pick = lo + (long long)i;
                break;
            }
        }
    }
    return __shfl_sync(full, pick, sel);
}

// Heat-bath decisions of a level are made either by lanes (one variable per
// thread, rounds of tpr variables) or by warps (one variable per warp, its
// candidates split over the lanes, rounds of tpr / 32 variables), whichever
// costs fewer candidate evaluations per thread for the level's width `w`:
// lane mode walks up to 3 n candidates (n = max u - l + 1; about n with the
// closed-form windows of float QUIO below 256 values), warp mode about 6 n / 32
// plus the fixed cost of a decision.  Every thread of a group takes the same
// choice.
__device__ __forceinline__ bool hb_warp_mode(int w, int tpr, uint32_t max_width, bool small_path) {
    const float n = (float)max_width + 1.f;
    if (n < 32.f) return false;
    const int W = tpr >> 5;
    const float lane_cost = (float)((w + tpr - 1) / tpr) * (small_path ? 1.f : 3.f) * n;
    const float warp_cost = (float)((w + W - 1) / W) * (6.f * n / 32.f + 160.f);
    return warp_cost < lane_cost;
}

// Float QUIO with at most 256 values: dE(dz) = dz (c1 + d dz), dz = v - z,
// c1 = f + 2 d z.  The minimum comes from the endpoints, dz = 0 and the
// integers around the vertex.  The kept window is derived in closed form: for
// d > 0 with the vertex vq inside the range every value with
// dE - dE_min <= C (C = the cut times T) satisfies d (dz - vq)^2 <= C + d/4, so
// vq -/+ sqrt(C/d + 1/4) brackets it; with the vertex outside the range dE is
// monotone over it and, by convexity, the window ends within C / slope of the
// minimising endpoint; for d <= 0 the window is the whole range.  Blocks of 16
// values counted from the window start (so every lane loops over its own
// window) are summed in registers; the pick scans the block sums and
// recomputes one block.
// weight 2^((dE_min - dE(dz)) b2), the exponent written as the polynomial
// A dz^2 + B dz + C with A = -b2 d, B = -b2 c1, C = b2 dE_min (Horner form)
__device__ __forceinline__ float quio_w(float dz, float A, float B, float C) {
    return ex2_ftz(fmaf(fmaf(A, dz, B), dz, C));
}

// The window only has to contain every value within the cut, and every bound
// below carries a margin of at least one value, so its arithmetic uses the
// fast approximate divide, reciprocal square root and logarithm (relative
// errors of a few ulp); the weights themselves are computed as elsewhere.
// `temp` is T = 1 / beta.
__device__ __forceinline__ long long heat_bath_quio_f32_small(float f, float d, long long z, long long lo,
                                                              uint32_t width, uint32_t xu, float beta, float temp) {
    const int n = (int)width + 1;
    const float zf = __int2float_rn((int)z);
    const float dz0 = __int2float_rn((int)(lo - z));
    const float c1 = fmaf(2.f * d, zf, f);
    const float dzn = dz0 + (float)width;
    const float e0 = dz0 * fmaf(d, dz0, c1), en = dzn * fmaf(d, dzn, c1);
    float mn = fminf(0.f, fminf(e0, en));
    const float C = (20.f + __logf((float)width + 1.f)) * temp;   // hb_cut(width) / beta
    float wlo = dz0, whi = dzn;
    if (d > 0.f) {
        const float vq = __fdividef(-c1, 2.f * d);
        if (vq > dz0 && vq < dzn) {
            const float q = floorf(vq), q1 = q + 1.f;
            mn = fminf(mn, fminf(q * fmaf(d, q, c1), q1 * fmaf(d, q1, c1)));
            const float h2 = __fdividef(C, d) + 0.25f;
            const float h = h2 * rsqrtf(h2) + 1.f;                  // sqrt(C / d + 1/4) + 1
            wlo = fmaxf(dz0, floorf(vq - h));
            whi = fminf(dzn, ceilf(vq + h));
        } else if (vq <= dz0) {      // increasing over the range: minimum at dz0
            const float slope = fmaf(d, fmaf(2.f, dz0, 1.f), c1);   // dE(dz0 + 1) - dE(dz0) > 0
            whi = fminf(dzn, dz0 + ceilf(__fdividef(C, slope)) + 1.f);
        } else {                      // decreasing: minimum at dzn
            const float slope = -fmaf(d, fmaf(2.f, dzn, -1.f), c1); // dE(dzn - 1) - dE(dzn) > 0
            wlo = fmaxf(dz0, dzn - ceilf(__fdividef(C, slope)) - 1.f);
        }
        if (!(wlo <= whi)) { wlo = dz0; whi = dzn; }   // non-finite slope etc.: whole range
    }
    const float b2 = beta * 1.4426950408889634f, mb = mn * b2;
    const float hA = -b2 * d, hB = -b2 * c1;
    const int kb0 = (int)(wlo - dz0) >> 4, kb1 = (int)(whi - dz0) >> 4;
    const int base = kb0 * 16;
    const int nrb = kb1 - kb0 + 1;
    const float dzb0 = dz0 + (float)base;
    // block sums in registers (the loops are unrolled, so bs[] is indexed by
    // constants); both loops stop after the window's nrb blocks
    float bs[16];
    float tot = 0.f;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        if (b >= nrb) break;
        float acc = 0.f;
        const float a0 = dzb0 + (float)(b * 16);
        if (base + b * 16 + 15 < n) {
            float w[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) w[j] = quio_w(a0 + (float)j, hA, hB, mb);
#pragma unroll
            for (int h = 8; h >= 1; h >>= 1)
#pragma unroll
                for (int j = 0; j < h; ++j) w[j] += w[j + h];
            acc = w[0];
        } else {
            const int cnt = n - (base + b * 16);
            for (int j = 0; j < cnt; ++j) acc += quio_w(a0 + (float)j, hA, hB, mb);
        }
        bs[b] = acc;
        tot += acc;
    }
    const float thr = unit_open_left(xu) * tot;
    float run = 0.f, before_last = 0.f;
    int sel = -1;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        if (b >= nrb) break;
        const float nxt = run + bs[b];
        if (nxt >= thr) {
            sel = b;
            break;
        }
        before_last = run;
        run = nxt;
    }
    if (sel < 0) {  // rounding left the threshold above the window: take its last block
        sel = nrb - 1;
        run = before_last;
    }
    // the chosen block: its weights first (independent exp2), then the
    // smallest value whose running sum reaches the threshold
    const int first = base + sel * 16;
    const int cnt = min(16, n - first);
    const float a0 = dz0 + (float)first;
    float w[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) w[j] = j < cnt ? quio_w(a0 + (float)j, hA, hB, mb) : 0.f;
    int pick = cnt - 1;
    bool found = false;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        run += w[j];
        const bool hit = !found && j < cnt && run >= thr;
        pick = hit ? j : pick;
        found = found || hit;
    }
    return lo + (long long)(first + pick);
}

// Multilinear variable, dE = a (v - z): P(i) proportional to exp(-lambda i) on
// i = 0..n-1, lambda = a beta; inverse transform of Eq. inverse_prob.  The pick
// is i = ceil(X) - 1 where X solves P_sum(X - 1) = Uc:
//   lambda > 0:  X = -log1p(Uc expm1(-lambda n)) / lambda
//   lambda < 0:  X = n - Y,  Y = -log1p((1 - Uc) expm1(-mu n)) / mu,  mu = -lambda,
//                so i = (n - 1) - floor(Y)
// (the second keeps the distance from the top, Y, as the computed quantity so
// that neither a cancellation nor the spacing of floats near n loses it).
__device__ __forceinline__ long long heat_bath_linear(float a, long long lo, uint32_t width, uint32_t xu,
                                                      float beta) {
    const float U = unit_open_left(xu);
    const float lam = a * beta;
    long long i;
    if (width < (1u << 24)) {
        const float n = (float)(width + 1u);
        if (lam == 0.f) {
            i = (long long)ceilf(U * n) - 1;
        } else if (lam > 0.f) {
            const float X = -log1pf(U * expm1f(-lam * n)) / lam;
            i = (long long)ceilf(X) - 1;
        } else {
            const float mu = -lam;
            const float Y = -log1pf((1.f - U) * expm1f(-mu * n)) / mu;
            i = (long long)width - (long long)floorf(Y);
        }
    } else {
        const double n = (double)width + 1.0, Ud = (double)U, l = (double)lam;
        if (l == 0.0) {
            i = (long long)ceil(Ud * n) - 1;
        } else if (l > 0.0) {
            i = (long long)ceil(-log1p(Ud * expm1(-l * n)) / l) - 1;
        } else {
            const double Y = -log1p((1.0 - Ud) * expm1(l * n)) / (-l);
            i = (long long)width - (long long)floor(Y);
        }
    }
    if (i < 0) i = 0;
    if (i > (long long)width) i = (long long)width;
    return lo + i;
}

// ------------------------------------------------------------------ cache recompute
// QUIO: f_k = lin_k + sum_j J_kj z_j (exact int64, or FP64 then cast to fp32).
// Returns this thread's share of E: sum_k z_k (lin_k + diag_k z_k) and
// sum_k z_k (f_k - lin_k) (twice the pair energy).
template <class F, class Z>
__device__ void quio_recompute(const DevModel& m, const Z* zs, F* cache, int t, int tpr, bool measure,
                               float& drift, typename Num<F>::Acc& e_ld, typename Num<F>::Acc& e_pair2) {
    for (int k = t; k < m.n; k += tpr) {
        const VarMeta mt = m.meta[k];
        const long long zk = (long long)mt.lo + (long long)zs[k];
        if constexpr (Num<F>::is_float) {
            double f = m.lin_d[k];
            for (int e = mt.link_begin; e < mt.link_begin + mt.link_len; ++e) {
                const int j = m.adj_col[e];
                const double w = m.adj_d ? m.adj_d[e] : (double)m.adj_f[e];
                // z_j fits int32 (model compiler): a 32-bit source conversion
                f += w * __int2double_rn(m.meta[j].lo + (int)zs[j]);
            }
            const float ff = (float)f;
            if (measure) drift = fmaxf(drift, (float)fabs((double)cache[k] - f));
            cache[k] = ff;
            e_ld += (double)zk * (m.lin_d[k] + m.diag_d[k] * (double)zk);
            e_pair2 += (double)zk * (f - m.lin_d[k]);
        } else {
            long long f = m.lin_i[k];
            for (int e = mt.link_begin; e < mt.link_begin + mt.link_len; ++e) {
                const int j = m.adj_col[e];
                f += m.adj_i[e] * ((long long)m.meta[j].lo + (long long)zs[j]);
            }
            cache[k] = f;
            e_ld += zk * (m.lin_i[k] + m.diag_i[k] * zk);
            e_pair2 += zk * (f - m.lin_i[k]);
        }
    }
}

// HUIO: a_k^(m) = J_{k..k} + sum over interaction terms t containing k with
// exponent m of J_t prod_{i in t, i != k} z_i^{e_i}.  Thread k owns its slots.
// Energy share: single-variable terms of the owned variables plus the
// interaction terms t = t0, t0 + tpr, ...
template <class F, class Z>
__device__ void huio_recompute(const DevModel& m, const Z* zs, F* cache, int t, int tpr, bool measure,
                               float& drift, typename Num<F>::Acc& e_self, typename Num<F>::Acc& e_terms) {
    using Acc = typename Num<F>::Acc;
    for (int k = t; k < m.n; k += tpr) {
        const VarMeta mt = m.meta[k];
        const long long zk = (long long)mt.lo + (long long)zs[k];
        const int base = m.slot_base[k];
        const uint64_t om = m.omega[k];
        const int nsl = __popcll(om);
        // start from the constants, accumulate interaction contributions
        Acc acc[8];
        const int nloc = nsl < 8 ? nsl : 8;
        for (int q = 0; q < nloc; ++q) {
            if constexpr (Num<F>::is_float) acc[q] = m.aconst_d[base + q];
            else acc[q] = m.aconst_i[base + q];
        }
        for (int q = nloc; q < nsl; ++q) {
            if constexpr (Num<F>::is_float) cache[base + q] = (F)m.aconst_d[base + q];
            else cache[base + q] = m.aconst_i[base + q];
        }
        for (int e = mt.link_begin; e < mt.link_begin + mt.link_len; ++e) {
            const int tt = m.inc_term[e];
            const int ek = m.inc_exp[e];
            Acc prod;
            if constexpr (Num<F>::is_float) prod = m.tcoef_d[tt];
            else prod = m.tcoef_i[tt];
            for (int p = m.term_ptr[tt]; p < m.term_ptr[tt + 1]; ++p) {
                const int v = m.mem_var[p];
                if (v == k) continue;
                const long long zv = (long long)m.meta[v].lo + (long long)zs[v];
                prod *= ipow<Acc>((Acc)zv, m.mem_exp[p]);
            }
            const int q = __popcll((om & ((1ull << ek) - 1ull)) >> 1);
            if (q < 8) acc[q] += prod;
            else cache[base + q] += (F)prod;
        }
        for (int q = 0; q < nloc; ++q) {
            if constexpr (Num<F>::is_float) {
                if (measure) drift = fmaxf(drift, (float)fabs((double)cache[base + q] - acc[q]));
                cache[base + q] = (float)acc[q];
            } else {
                cache[base + q] = acc[q];
            }
        }
        // single-variable terms' energy: sum_m aconst z^m
        uint64_t msk = om >> 1;
        Acc pz = 1;
        int q = 0;
        while (msk) {
            pz *= (Acc)zk;
            if (msk & 1ull) {
                if constexpr (Num<F>::is_float) e_self += m.aconst_d[base + q] * pz;
                else e_self += m.aconst_i[base + q] * pz;
                ++q;
            }
            msk >>= 1;
        }
    }
    for (int tt = t; tt < m.n_iterms; tt += tpr) {
        Acc prod;
        if constexpr (Num<F>::is_float) prod = m.tcoef_d[tt];
        else prod = m.tcoef_i[tt];
        for (int p = m.term_ptr[tt]; p < m.term_ptr[tt + 1]; ++p) {
            const int v = m.mem_var[p];
            const long long zv = (long long)m.meta[v].lo + (long long)zs[v];
            prod *= ipow<Acc>((Acc)zv, m.mem_exp[p]);
        }
        e_terms += prod;
    }
}

// ------------------------------------------------------------------ cache update
// QUIO (Sect. 3.2): z_s += dz changes f_j by J_sj dz for every neighbour j.
// Strided form, used by the cooperative path.
template <class F>
__device__ __forceinline__ void quio_update_range(const DevModel& m, F* cache, int begin, int end, int stride,
                                                  long long dz) {
    if constexpr (Num<F>::is_float) {
        const float d = (float)(int)dz;
        for (int e = begin; e < end; e += stride) atomic_add_field(cache + m.adj_col[e], __ldg(m.adj_f + e) * d);
    } else {
        for (int e = begin; e < end; e += stride) atomic_add_field(cache + m.adj_col[e], m.adj_i[e] * dz);
    }
}

// One thread, whole row: rows are padded to multiples of 4 entries and start on
// 16-byte boundaries, so 16 entries arrive in one round of vector loads that is
// issued before any of their atomics.
template <class F>
__device__ __forceinline__ void quio_update_row(const DevModel& m, F* cache, int begin, int len, long long dz) {
    const int4* cp = reinterpret_cast<const int4*>(m.adj_col + begin);
    const int nq = (len + 3) >> 2;
    if constexpr (Num<F>::is_float) {
        const float d = (float)(int)dz;
        const float4* vp = reinterpret_cast<const float4*>(m.adj_f + begin);
        for (int q0 = 0; q0 < nq; q0 += 4) {
            int4 c[4];
            float4 w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (q0 + u < nq) {
                    c[u] = __ldg(cp + q0 + u);
                    w[u] = __ldg(vp + q0 + u);
                }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = 4 * (q0 + u);
                if (e + 0 < len) atomic_add_field(cache + c[u].x, w[u].x * d);
                if (e + 1 < len) atomic_add_field(cache + c[u].y, w[u].y * d);
                if (e + 2 < len) atomic_add_field(cache + c[u].z, w[u].z * d);
                if (e + 3 < len) atomic_add_field(cache + c[u].w, w[u].w * d);
            }
        }
    } else {
        const longlong2* vp = reinterpret_cast<const longlong2*>(m.adj_i + begin);
        for (int q0 = 0; q0 < nq; q0 += 2) {
            int4 c[2];
            longlong2 w[4];
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (q0 + u < nq) {
                    c[u] = __ldg(cp + q0 + u);
                    w[2 * u] = __ldg(vp + 2 * (q0 + u));
                    w[2 * u + 1] = __ldg(vp + 2 * (q0 + u) + 1);
                }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int e = 4 * (q0 + u);
                if (e + 0 < len) atomic_add_field(cache + c[u].x, w[2 * u].x * dz);
                if (e + 1 < len) atomic_add_field(cache + c[u].y, w[2 * u].y * dz);
                if (e + 2 < len) atomic_add_field(cache + c[u].z, w[2 * u + 1].x * dz);
                if (e + 3 < len) atomic_add_field(cache + c[u].w, w[2 * u + 1].y * dz);
            }
        }
    }
}

// HUIO (Eq. energy_diff_upd): for every interaction term t containing s with
// exponent e_s, and every other member k with exponent e_k,
//   a_k^(e_k) += J_t ((z_s')^{e_s} - z_s^{e_s}) prod_{i in t \ {k, s}} z_i^{e_i}.
// One incidence e of s: the term's members (at most kTermRegs) are read once
// into registers through the read-only path, the products over the other
// members come from prefix and suffix products, and the model loads of
// consecutive incidences do not wait on the previous incidence's atomics.
constexpr int kTermRegs = 8;

template <class F, class Z>
__device__ __forceinline__ void huio_update_one(const DevModel& m, const Z* zs, F* cache, int s, int e,
                                                long long z_old, long long z_new) {
    const int4* rec = reinterpret_cast<const int4*>(m.inc_rec) + 3 * (size_t)e;
    const int4 r0 = __ldg(rec);
    if (r0.z >= 0) {
        // term of at most 4 members: its record holds the other members and
        // their slots, so the z values, bounds and coefficient load together
        const int4 r1 = __ldg(rec + 1), r2 = __ldg(rec + 2);
        const int no = r0.z, es = r0.y, ep = r1.w;
        const int vv[3] = {r1.x, r1.y, r1.z};
        const int sl[3] = {r2.x, r2.y, r2.z};
        F base;
        if constexpr (Num<F>::is_float)
            base = Coef<float>::tcoef(m, r0.x) * (ipow<float>((float)z_new, es) - ipow<float>((float)z_old, es));
        else base = __ldg(m.tcoef_i + r0.x) * (ipow<long long>(z_new, es) - ipow<long long>(z_old, es));
        F zp[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            zp[i] = F(1);
            if (i < no) {
                const long long zv = (long long)__ldg(&m.meta[vv[i]].lo) + (long long)zs[vv[i]];
                const int ex = (ep >> (8 * i)) & 0xFF;
                if constexpr (Num<F>::is_float) zp[i] = ipow<float>((float)zv, ex);
                else zp[i] = ipow<long long>(zv, ex);
            }
        }
        // member i receives base times the other members' powers
        if (no > 0) atomic_add_field(cache + sl[0], base * zp[1] * zp[2]);
        if (no > 1) atomic_add_field(cache + sl[1], base * zp[0] * zp[2]);
        if (no > 2) atomic_add_field(cache + sl[2], base * zp[0] * zp[1]);
        return;
    }
    const int tt = r0.x;
    const int es = r0.y;
    const int p0 = __ldg(m.term_ptr + tt), p1 = __ldg(m.term_ptr + tt + 1);
    const int nm = p1 - p0;
    F base;
    if constexpr (Num<F>::is_float) base = Coef<float>::tcoef(m, tt) * (ipow<float>((float)z_new, es) - ipow<float>((float)z_old, es));
    else base = __ldg(m.tcoef_i + tt) * (ipow<long long>(z_new, es) - ipow<long long>(z_old, es));
    if (nm <= kTermRegs) {
        int var[kTermRegs], ex[kTermRegs];
        F zp[kTermRegs];
#pragma unroll
        for (int i = 0; i < kTermRegs; ++i) {
            if (i < nm) {
                var[i] = __ldg(m.mem_var + p0 + i);
                ex[i] = __ldg(m.mem_exp + p0 + i);
            }
        }
#pragma unroll
        for (int i = 0; i < kTermRegs; ++i) {
            zp[i] = F(1);
            if (i < nm && var[i] != s) {
                const long long zv = (long long)__ldg(&m.meta[var[i]].lo) + (long long)zs[var[i]];
                if constexpr (Num<F>::is_float) zp[i] = ipow<float>((float)zv, ex[i]);
                else zp[i] = ipow<long long>(zv, ex[i]);
            }
        }
        // suffix products: suf[i] = prod_{j >= i} zp[j]
        F suf[kTermRegs + 1];
        suf[kTermRegs] = F(1);
#pragma unroll
        for (int i = kTermRegs - 1; i >= 0; --i) suf[i] = suf[i + 1] * zp[i];
        F pre = base;
#pragma unroll
        for (int i = 0; i < kTermRegs; ++i) {
            if (i < nm && var[i] != s) {
                const int k = var[i];
                const uint64_t om = __ldg(m.omega + k);
                const int q = __popcll((om & ((1ull << ex[i]) - 1ull)) >> 1);
                atomic_add_field(cache + __ldg(m.slot_base + k) + q, pre * suf[i + 1]);
            }
            pre *= zp[i];
        }
        return;
    }
    for (int pk = p0; pk < p1; ++pk) {
        const int k = __ldg(m.mem_var + pk);
        if (k == s) continue;
        F prod = base;
        for (int pi = p0; pi < p1; ++pi) {
            const int v = __ldg(m.mem_var + pi);
            if (v == s || v == k) continue;
            const long long zv = (long long)__ldg(&m.meta[v].lo) + (long long)zs[v];
            if constexpr (Num<F>::is_float) prod *= ipow<float>((float)zv, __ldg(m.mem_exp + pi));
            else prod *= ipow<long long>(zv, __ldg(m.mem_exp + pi));
        }
        const uint64_t om = __ldg(m.omega + k);
        const int ek = __ldg(m.mem_exp + pk);
        const int q = __popcll((om & ((1ull << ek) - 1ull)) >> 1);
        atomic_add_field(cache + __ldg(m.slot_base + k) + q, prod);
    }
}

template <class F, class Z>
__device__ __forceinline__ void huio_update_range(const DevModel& m, const Z* zs, F* cache, int s, int begin,
                                                  int end, int stride, long long z_old, long long z_new) {
    for (int e = begin; e < end; e += stride) huio_update_one<F, Z>(m, zs, cache, s, e, z_old, z_new);
}

// Field update of a level's only variable (no other writer): rounded product,
// then rounded sum, at every call site, so that every schedule of the same
// updates gives the same fp32 fields.
__device__ __forceinline__ void solo_add(float* c, float w, long long dz) {
    *c = __fadd_rn(*c, __fmul_rn(w, (float)(int)dz));
}
__device__ __forceinline__ void solo_add(long long* c, long long w, long long dz) { *c += w * dz; }

// ------------------------------------------------------------------ reductions
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the replica's threads; result valid in every thread.
template <class T>
__device__ T group_sum(T v, T* red, int t, int tpr, int bar_id) {
    v = warp_sum(v);
    const int w = t >> 5;
    named_bar(bar_id, tpr);  // red[] free
    if ((t & 31) == 0) red[w] = v;
    named_bar(bar_id, tpr);
    T tot = T(0);
    for (int i = 0; i < (tpr >> 5); ++i) tot += red[i];
    return tot;
}

// ------------------------------------------------------------------ best state
// Optional best state at sweep ends, called by every thread of the group with
// the sweep's energy `tot` (the same in every thread): the best energy so far
// lives in the output, where the previous sweep, or the group that ran the
// replica's earlier sweeps, left it (`first`: this run has none yet).  A
// strictly lower energy replaces it and the state is copied, so the earliest
// sweep wins ties.  Kept out of line: it runs only when the caller asks for
// best states.
template <class Acc, class Z>
__device__ __noinline__ void keep_best(const SweepArgs& a, const Z* zs, int r, int t, int tpr, int bar_id, Acc tot,
                                       bool first) {
    Acc* bst = reinterpret_cast<Acc*>(a.best_energies) + r;
    const bool better = first || tot < __ldcg(bst);
    named_bar(bar_id, tpr);   // every thread has read the old value before thread 0 replaces it
    if (!better) return;
    if (t == 0) *bst = tot;
    int32_t* dst = a.best_states + (size_t)r * a.m.n;
    for (int k = t; k < a.m.n; k += tpr) dst[k] = (int32_t)((long long)a.m.meta[k].lo + (long long)zs[k]);
    named_bar(bar_id, tpr);   // every thread has read zs before the next sweep changes it
}

// ------------------------------------------------------------------ one replica
// Sweeps [s0, s1) of the SA run of replica r (Sect. 3.1) by the `tpr` threads
// of one group; `base` is the group's state region (shared or global memory).
// A run that starts at s0 = 0 draws (or takes) the initial state and builds
// the caches; otherwise it restores the state and the per-thread accumulators
// that the run of sweeps [0, s0) saved at `restore`.  A run that ends at
// s1 = S writes the outputs; otherwise it saves its state at `save` (layout:
// bytes [0, off_ctl) of the state region, then per thread the energy
// accumulator, the change count and the refresh drift, 24 bytes each).
template <class F, class Z, int RULE, int KIND>
__device__ __forceinline__ void replica_body(const SweepArgs& a, const int slot, const int t, const int r,
                                             uint8_t* base, const int s0 = 0, int s1 = -1,
                                             const uint8_t* restore = nullptr, uint8_t* save = nullptr) {
    using Acc = typename Num<F>::Acc;
    const DevModel& m = a.m;
    const int bar_id = 1 + slot;
    const int tpr = a.tpr;
    if (s1 < 0) s1 = a.S;
    Z* zs = reinterpret_cast<Z*>(base + a.off_z);
    F* cache = reinterpret_cast<F*>(base + a.off_cache);
    // [0..2] list counters, [3] flattened length, [4..27] two results of speculative windows
    int* ctl = reinterpret_cast<int*>(base + a.off_ctl);
    // [cap][6]: variable k, z_old, z_new, link_begin, link_len, prefix of the
    // flattened (entry, link) pairs
    int* list = reinterpret_cast<int*>(base + a.off_list);
    Acc* red = reinterpret_cast<Acc*>(base + a.off_red);

    if (t == 0) { ctl[0] = 0; ctl[1] = 0; ctl[2] = 0; }
    // level boundaries, staged on chip when the table is small
    int* lvl_s = a.off_lvl >= 0 ? reinterpret_cast<int*>(base + a.off_lvl) : nullptr;
    if (lvl_s)
        for (int L = t; L <= m.n_levels; L += tpr) lvl_s[L] = __ldg(m.lvl_ptr + L);
    float drift = 0.f;
    Acc eacc;
    unsigned long long changes = 0;
    if (restore == nullptr) {
        // ---- random initial state (Sect. 3.1), or the caller's
        for (int k = t; k < m.n; k += tpr) {
            const VarMeta mt = m.meta[k];
            uint32_t off;
            if (a.init_states) {
                off = (uint32_t)((long long)a.init_states[(size_t)r * m.n + k] - (long long)mt.lo);
            } else {
                const Words4 x = philox4x32_10((uint32_t)k, 0xFFFFFFFFu, (uint32_t)r, a.inst, a.key0, a.key1);
                off = pick_below(x.x0, mt.width + 1u);
            }
            zs[k] = (Z)off;
        }
        named_bar(bar_id, tpr);
        Acc e1 = 0, e2 = 0;
        if constexpr (KIND == KIND_QUIO) quio_recompute<F, Z>(m, zs, cache, t, tpr, false, drift, e1, e2);
        else huio_recompute<F, Z>(m, zs, cache, t, tpr, false, drift, e1, e2);
        // per-thread energy accumulator: this thread's share of E(z_init)
        if constexpr (KIND == KIND_QUIO) {
            // pair share is counted twice over the replica; halve after the sum
            Acc pair2 = group_sum<Acc>(e2, red, t, tpr, bar_id);
            eacc = e1 + (t == 0 ? pair2 / 2 : Acc(0));
        } else {
            eacc = e1 + e2;
            named_bar(bar_id, tpr);
        }
        if (t == 0) {
            if constexpr (Num<F>::is_float) eacc += m.const_d;
            else eacc += m.const_i;
        }
    } else {
        // ---- state of sweeps [0, s0), saved by another group
        const int nq = a.off_ctl / 16;
        const uint4* src = reinterpret_cast<const uint4*>(restore);
        uint4* dst = reinterpret_cast<uint4*>(base);
        for (int q = t; q < nq; q += tpr) dst[q] = __ldcg(src + q);
        const uint8_t* acc = restore + a.off_ctl + (size_t)t * 24;
        const unsigned long long e_bits = __ldcg(reinterpret_cast<const unsigned long long*>(acc));
        eacc = *reinterpret_cast<const Acc*>(&e_bits);
        changes = __ldcg(reinterpret_cast<const unsigned long long*>(acc + 8));
        drift = __ldcg(reinterpret_cast<const float*>(acc + 16));
        named_bar(bar_id, tpr);
    }

    float dacc = 0.f;  // float models: energy changes since the last fold into eacc
    int gl3 = 0;  // level counter mod 3: which cooperative-list counter is live

    // Decision for one record (reads replica state only).  With `wmode` the 32
    // lanes of a warp call it together for the same record (heat bath only).
    auto decide = [&](const LevelRec& rc, int s, float beta, float temp, float ratio, long long& z, long long& v,
                      F& de, bool wmode) {
        const int k = rc.k;
        const long long lo = rc.lo;
        const long long zo = (long long)zs[k];
        z = lo + zo;
        v = z;
        de = F(0);
        if (rc.width == 0) return;
        const Words4 x = philox4x32_10((uint32_t)k, (uint32_t)s, (uint32_t)r, a.inst, a.key0, a.key1);
        VarView<F, KIND> vv;
        if constexpr (KIND == KIND_QUIO) {
            vv.f = cache[k];
            if constexpr (Num<F>::is_float) vv.d = __uint_as_float(rc.aux0);
            else vv.d = (long long)(((unsigned long long)rc.aux1 << 32) | rc.aux0);
        } else {
            vv.a = cache + rc.slot_base;
            vv.omega = ((uint64_t)rc.aux1 << 32) | rc.aux0;
        }
        const long long hi = lo + (long long)rc.width;
        if constexpr (RULE == RULE_HEAT_BATH) {
            if (vv.linear()) {
                v = heat_bath_linear(Num<F>::to_f(vv.lin_coef()), lo, rc.width, x.x0, beta);
            } else if (wmode) {
                v = heat_bath_warp<F, KIND>(vv, z, lo, rc.width, x.x0, beta, t & 31);
            } else {
                bool done = false;
                if constexpr (Num<F>::is_float && KIND == KIND_QUIO) {
                    if (rc.width < 256u && lo > -(1 << 22) && hi < (1 << 22)) {
                        v = heat_bath_quio_f32_small((float)vv.f, (float)vv.d, z, lo, rc.width, x.x0, beta, temp);
                        done = true;
                    }
                }
                if (!done) v = heat_bath_general<F, KIND>(vv, z, lo, rc.width, x.x0, beta);
            }
            if (v != z) de = vv.delta(z, v);
        } else {
            long long prop;
            if (RULE == RULE_OPT && unit_open_right(x.x2) < ratio) {
                prop = opt_argmin<F, KIND>(vv, z, lo, hi);
            } else {
                const uint32_t j = pick_below(x.x0, rc.width);
                prop = lo + (long long)(j >= (uint32_t)zo ? j + 1u : j);
            }
            const F dprop = vv.delta(z, prop);
            if (metropolis_accept<F>(dprop, x.x1, beta)) {
                v = prop;
                de = dprop;
            }
        }
    };
    // Applies a decision: state, energy, counters and the neighbours' caches
    // (inline for short incidence lists, else through the cooperative list).
    auto apply = [&](const LevelRec& rc, int s, long long z, long long v, F de, int* cnt_now, bool& coop) {
        const int k = rc.k;
        if (v != z) {
            zs[k] = (Z)(v - (long long)rc.lo);
            if constexpr (Num<F>::is_float) dacc += (float)de;   // folded into eacc at refreshes
            else eacc += (Acc)de;
            ++changes;
            const int len = rc.link_len;
            bool inline_upd = len <= a.heavy_links;
            if (!inline_upd) {
                const int idx = atomicAdd(cnt_now, 1);
                if (idx < a.list_cap) {
                    int* e = list + 6 * idx;
                    e[0] = k;
                    e[1] = (int)z;
                    e[2] = (int)v;
                    e[3] = rc.link_begin;
                    e[4] = len;
                } else {
                    inline_upd = true;
                }
            }
            if (inline_upd) {
                if constexpr (KIND == KIND_QUIO)
                    coop = true;   // the warp updates this row together (below)
                else
                    huio_update_range<F, Z>(m, zs, cache, k, rc.link_begin, rc.link_begin + len, 1, z, v);
            }
        }
        if (a.trace != nullptr && r < a.trace_R) a.trace[((size_t)s * a.trace_R + r) * m.n + k] = (int32_t)v;
    };
    auto load_rec = [&](int i) -> LevelRec {
        const int4* p = reinterpret_cast<const int4*>(m.lvl_rec + i);
        const int4 x0 = __ldg(p), x1 = __ldg(p + 1);
        LevelRec q;
        q.k = x0.x; q.lo = x0.y; q.width = (uint32_t)x0.z; q.link_begin = x0.w;
        q.link_len = x1.x; q.slot_base = x1.y; q.aux0 = (uint32_t)x1.z; q.aux1 = (uint32_t)x1.w;
        return q;
    };

    auto lvl_at = [&](int L) -> int { return lvl_s ? lvl_s[L] : __ldg(m.lvl_ptr + L); };
    // prefetch into L1 the records this thread will read in level L
    auto prefetch_level = [&](int L) {
        const int b0 = lvl_at(L), b1 = lvl_at(L + 1);
        for (int i = b0 + t; i < b1; i += tpr) prefetch_l1(m.lvl_rec + i);
    };
    prefetch_level(0);
    int win = 0;   // speculative windows run so far (their result slots alternate)
    for (int s = s0; s < s1; ++s) {
        const float beta = __ldg(a.beta + s);
        const float temp = 1.f / beta;
        const float ratio = __ldg(a.ratio + s);
        for (int L = 0; L < m.n_levels; ++L) {
            int* cnt_now = ctl + gl3;
            if (t == 0) ctl[gl3 == 2 ? 0 : gl3 + 1] = 0;
            const int lb = lvl_at(L), le = lvl_at(L + 1);
            // heat bath over wide ranges gives a narrow level's variables a warp each
            bool wmode = false;
            if constexpr (RULE == RULE_HEAT_BATH)
                wmode = hb_warp_mode(le - lb, tpr, m.max_width,
                                     Num<F>::is_float && KIND == KIND_QUIO && m.max_width < 256u);
            // (QUIO only, and neither float heat bath nor heat bath in warp mode:
            // second inlined copies of their decision or update code would make
            // the kernel spill registers)
            constexpr bool kSpeculative = KIND == KIND_QUIO && !(RULE == RULE_HEAT_BATH && Num<F>::is_float);
            if constexpr (kSpeculative) if (a.speculate && le - lb == 1 && !wmode) {
                // ---- a run of single-variable levels (every level of a complete
                // graph), decided by the lanes of warp 0, up to 32 levels at a
                // time, lane i deciding level L + i.  Every decision before the first one that changes
                // its variable saw the state of the level-by-level order, since
                // nothing changed before it, and so did that one; the group then
                // updates that variable's neighbours and the next window starts
                // after it.  Results equal those of the level-by-level order; the
                // energy change and the count go to thread 0 as they do there.
                int* res = ctl + 4 + 12 * (win & 1);   // {k or -1, levels done, row begin, row length,
                                                      //  z_old (2), z_new (2), dE (2)}
                if (t < 32) {
                    const int lane = t;
                    const int Li = L + lane;
                    int idx = 0;
                    bool single = false;
                    if (Li < m.n_levels) {
                        idx = lvl_at(Li);
                        single = lvl_at(Li + 1) - idx == 1;
                    }
                    const unsigned multi = __ballot_sync(0xffffffffu, !single);
                    const int w = multi ? __ffs(multi) - 1 : 32;   // >= 1: level L holds one variable
                    long long zz = 0, vv2 = 0;
                    F d2 = F(0);
                    LevelRec rc{};
                    int p = w;           // levels decided without a change
                    bool chg = false;    // level L + p changed its variable
                    if (lane < w) {
                        rc = load_rec(idx);
                        decide(rc, s, beta, temp, ratio, zz, vv2, d2, false);
                    }
                    {
                        const unsigned c = __ballot_sync(0xffffffffu, lane < w && vv2 != zz);
                        if (c) {
                            p = __ffs(c) - 1;
                            chg = true;
                        }
                        if (a.trace != nullptr && r < a.trace_R && (lane < p || (chg && lane == p)))
                            a.trace[((size_t)s * a.trace_R + r) * m.n + rc.k] = (int32_t)vv2;
                        // the changing lane's decision goes to lane 0
                        if (chg) {
                            const int k2 = __shfl_sync(0xffffffffu, rc.k, p);
                            const int lo2 = __shfl_sync(0xffffffffu, rc.lo, p);
                            const int b2 = __shfl_sync(0xffffffffu, rc.link_begin, p);
                            const int l2 = __shfl_sync(0xffffffffu, rc.link_len, p);
                            zz = __shfl_sync(0xffffffffu, zz, p);
                            vv2 = __shfl_sync(0xffffffffu, vv2, p);
                            d2 = __shfl_sync(0xffffffffu, d2, p);
                            rc.k = k2;
                            rc.lo = lo2;
                            rc.link_begin = b2;
                            rc.link_len = l2;
                        }
                    }
                    if (lane == 0) {
                        res[0] = chg ? rc.k : -1;
                        res[1] = chg ? p + 1 : w;
                        if (chg) {
                            zs[rc.k] = (Z)(vv2 - (long long)rc.lo);
                            res[2] = rc.link_begin;
                            res[3] = rc.link_len;
                            *reinterpret_cast<long long*>(res + 4) = zz;
                            *reinterpret_cast<long long*>(res + 6) = vv2;
                            *reinterpret_cast<F*>(res + 8) = d2;
                        }
                    }
                }
                named_bar(bar_id, tpr);
                const int kk = res[0];
                if (kk >= 0) {
                    const int rb = res[2], rl = res[3];
                    const long long zold = *reinterpret_cast<const long long*>(res + 4);
                    const long long znew = *reinterpret_cast<const long long*>(res + 6);
                    if (t == 0) {
                        if constexpr (Num<F>::is_float) dacc += (float)*reinterpret_cast<const F*>(res + 8);
                        else eacc += (Acc)*reinterpret_cast<const F*>(res + 8);
                        ++changes;
                    }
                    if (m.dense_rows) {
                        // row kk lists every j != kk in order: its columns need no reads
                        for (int e = t; e < rl; e += tpr)
                            solo_add(cache + e + (e >= kk ? 1 : 0), Coef<F>::adj(m, rb + e), znew - zold);
                    } else {
                        for (int e = rb + t; e < rb + rl; e += tpr)
                            solo_add(cache + __ldg(m.adj_col + e), Coef<F>::adj(m, e), znew - zold);
                    }
                    named_bar(bar_id, tpr);
                }
                L += res[1] - 1;
                ++win;
                gl3 = gl3 == 2 ? 0 : gl3 + 1;
                continue;
            }
            // the next level (the first level of the next sweep after the last)
            if (L + 1 < m.n_levels) prefetch_level(L + 1);
            else if (s + 1 < a.S) prefetch_level(0);
            // every thread of a warp runs the same number of rounds, so that the
            // warp can share the neighbour updates of its accepting lanes; heat
            // bath over wide ranges or narrow levels gives each variable a warp
            const int lane = t & 31;
            const bool solo = le - lb == 1;
            const int per_round = wmode ? (tpr >> 5) : tpr;
            const int slot_i = wmode ? (t >> 5) : t;
            const int rounds = (le - lb + per_round - 1) / per_round;
            for (int rd = 0; rd < rounds; ++rd) {
                const int i = lb + slot_i + rd * per_round;
                bool coop = false;
                int rb = 0, rl = 0;
                long long rdz = 0;
                if (i < le) {
                    const LevelRec rc = load_rec(i);
                    long long zz, vv2;
                    F d2;
                    decide(rc, s, beta, temp, ratio, zz, vv2, d2, wmode);
                    if (!wmode || lane == 0) {
                        apply(rc, s, zz, vv2, d2, cnt_now, coop);
                        rb = rc.link_begin;
                        rl = rc.link_len;
                        rdz = vv2 - zz;
                    }
                }
                if constexpr (KIND == KIND_QUIO) {
                    // Sect. 3.2 update of the accepted rows (coalesced row reads,
                    // parallel atomics)
                    unsigned pend = __ballot_sync(0xffffffffu, coop);
                    if (__popc(pend) > 4) {
                        // many accepting lanes: each updates its own row
                        if (coop) quio_update_row<F>(m, cache, rb, rl, rdz);
                        pend = 0;
                    }
                    // up to 4 accepting lanes: their rows are walked together, one
                    // entry per lane, with every row's loads issued before the
                    // atomics, so that the L2 latency is paid once per round
                    if (pend) {
                        int b4[4], l4[4], lmax = 0;
                        long long dz4[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int src = pend ? __ffs(pend) - 1 : 0;
                            const bool on = pend != 0u;
                            pend &= pend - 1;
                            b4[j] = __shfl_sync(0xffffffffu, rb, src);
                            l4[j] = on ? __shfl_sync(0xffffffffu, rl, src) : 0;
                            dz4[j] = __shfl_sync(0xffffffffu, rdz, src);
                            lmax = max(lmax, l4[j]);
                        }
                        for (int e0 = 0; e0 < lmax; e0 += 32) {
                            int col4[4];
                            F w4[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                if (e0 + lane < l4[j]) {
                                    col4[j] = __ldg(m.adj_col + b4[j] + e0 + lane);
                                    w4[j] = Coef<F>::adj(m, b4[j] + e0 + lane);
                                }
                            }
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                if (e0 + lane < l4[j]) {
                                    // a level's only variable: its row's columns are
                                    // distinct and nothing else touches the cache now
                                    if (solo) {
                                        solo_add(cache + col4[j], w4[j], dz4[j]);
                                    } else {
                                        F inc;
                                        if constexpr (Num<F>::is_float) inc = w4[j] * (float)(int)dz4[j];
                                        else inc = w4[j] * dz4[j];
                                        atomic_add_field(cache + col4[j], inc);
                                    }
                                }
                            }
                        }
                    }
                }
            }
            named_bar(bar_id, tpr);
            const int cnt = *cnt_now;
            if (cnt > 0) {
                // cooperative updates: every thread takes the next (entry, link)
                // pair; entry h owns links [pre_h, pre_h + len_h) of the flattened list
                const int nl = cnt < a.list_cap ? cnt : a.list_cap;
                int* total = ctl + 3;
                if (t == 0) {
                    int run = 0;
                    for (int h = 0; h < nl; ++h) {
                        list[6 * h + 5] = run;
                        run += list[6 * h + 4];
                    }
                    *total = run;
                }
                named_bar(bar_id, tpr);
                const int W = *total;
                int h = 0;
                for (int w = t; w < W; w += tpr) {
                    // largest h with pre_h <= w (w only grows: continue from the last h)
                    while (h + 1 < nl && list[6 * (h + 1) + 5] <= w) ++h;
                    const int* ent = list + 6 * h;
                    const int e = ent[3] + (w - ent[5]);
                    const long long zold = ent[1], znew = ent[2];
                    if constexpr (KIND == KIND_QUIO) {
                        if (solo) {   // one row, distinct columns: no atomics needed
                            solo_add(cache + m.adj_col[e], Coef<F>::adj(m, e), znew - zold);
                        } else {
                            quio_update_range<F>(m, cache, e, e + 1, 1, znew - zold);
                        }
                    } else {
                        huio_update_range<F, Z>(m, zs, cache, ent[0], e, e + 1, 1, zold, znew);
                    }
                }
                named_bar(bar_id, tpr);
            }
            gl3 = gl3 == 2 ? 0 : gl3 + 1;
        }
        // ---- FP64 refresh of float fields and energy
        if constexpr (Num<F>::is_float) {
            eacc += (double)dacc;
            dacc = 0.f;
            const bool last = (s + 1 == a.S);
            if (last || (a.refresh_interval > 0 && (s + 1) % a.refresh_interval == 0)) {
                Acc f1 = 0, f2 = 0;
                if constexpr (KIND == KIND_QUIO) {
                    quio_recompute<F, Z>(m, zs, cache, t, tpr, true, drift, f1, f2);
                    Acc pair2 = group_sum<Acc>(f2, red, t, tpr, bar_id);
                    eacc = f1 + (t == 0 ? pair2 / 2 : Acc(0));
                } else {
                    huio_recompute<F, Z>(m, zs, cache, t, tpr, true, drift, f1, f2);
                    eacc = f1 + f2;
                    named_bar(bar_id, tpr);
                }
                if (t == 0) eacc += m.const_d;
            }
        }
        if (a.energy_trace != nullptr || a.best_states != nullptr) {
            const Acc tot = group_sum<Acc>(eacc, red, t, tpr, bar_id);   // the same in every thread
            if (a.energy_trace != nullptr && t == 0) reinterpret_cast<Acc*>(a.energy_trace)[(size_t)s * a.R + r] = tot;
            if (a.best_states != nullptr)
                keep_best<Acc, Z>(a, zs, r, t, tpr, bar_id, tot, s == s0 && restore == nullptr);
        }
    }

    if (save != nullptr) {
        // ---- hand the state of sweeps [0, s1) to the group that runs the rest
        named_bar(bar_id, tpr);
        const int nq = a.off_ctl / 16;
        const uint4* src = reinterpret_cast<const uint4*>(base);
        uint4* dst = reinterpret_cast<uint4*>(save);
        for (int q = t; q < nq; q += tpr) dst[q] = src[q];
        uint8_t* acc = save + a.off_ctl + (size_t)t * 24;
        *reinterpret_cast<Acc*>(acc) = eacc;
        *reinterpret_cast<unsigned long long*>(acc + 8) = changes;
        *reinterpret_cast<float*>(acc + 16) = drift;
        return;
    }

    // ---- outputs
    const Acc etot = group_sum<Acc>(eacc, red, t, tpr, bar_id);
    const unsigned long long ctot = group_sum<unsigned long long>(changes, reinterpret_cast<unsigned long long*>(red), t, tpr, bar_id);
    for (int k = t; k < m.n; k += tpr)
        a.out_states[(size_t)r * m.n + k] = (int32_t)((long long)m.meta[k].lo + (long long)zs[k]);
    if (t == 0) {
        reinterpret_cast<Acc*>(a.out_energies)[r] = etot;
        if (a.out_accepts) a.out_accepts[r] = ctot;
    }
    if constexpr (Num<F>::is_float) {
        if (a.drift_bits != nullptr) {
            float dmax = drift;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
            if ((t & 31) == 0) atomicMax(a.drift_bits, __float_as_uint(dmax));
        }
    }
}

// ------------------------------------------------------------------ kernels
// One instance: replica blockIdx.x * rpc + slot per thread group.
template <class F, class Z, int RULE, int KIND, bool SMEM>
__global__ void __launch_bounds__(512, 1) sweep_kernel(const SweepArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int slot = threadIdx.x / a.tpr;
    const int t = threadIdx.x - slot * a.tpr;
    const int r = blockIdx.x * a.rpc + slot;
    if (slot >= a.rpc || r >= a.R) return;
    uint8_t* base = SMEM ? (smem_raw + (size_t)slot * (size_t)a.rep_bytes) : (a.gstate + (size_t)r * (size_t)a.rep_bytes);
    replica_body<F, Z, RULE, KIND>(a, slot, t, r, base);
}

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Upper bound on the polls of a handoff flag (each followed by a ~256 ns
// sleep).  The awaited chunk waits only on chunks claimed before it, so the
// bound only matters if the launch was not co-resident.
constexpr unsigned long long kHandoffSpinLimit = 1ull << 32;

// Time-sliced run of R replicas on the thread groups of a cooperative grid
// (every block resident at once): the groups claim (replica, chunk) tasks in
// chunk-major order (see slice_chunk_sweeps); a chunk after the first waits
// (bounded) until its replica's previous chunk has saved its state, restores
// it, runs its sweeps and saves the state for the next chunk.  Per-replica
// results equal those of sweep_kernel: every chunk draws the same Philox
// counters and the saved state includes the per-thread accumulators.
template <class F, class Z, int RULE, int KIND>
__global__ void __launch_bounds__(512, 1) sweep_sliced_kernel(const SweepArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ int task_s[16][2];
    const int slot = threadIdx.x / a.tpr;
    const int t = threadIdx.x - slot * a.tpr;
    if (slot >= a.rpc) return;
    const int bar_id = 1 + slot;
    uint8_t* base = smem_raw + (size_t)slot * (size_t)a.rep_bytes;
    const int32_t K = slice_chunk_sweeps(a.S);
    const int32_t C = (a.S + K - 1) / K;
    const unsigned int n_tasks = (unsigned int)a.R * (unsigned int)C;
    for (;;) {
        named_bar(bar_id, a.tpr);   // the previous task is done with the state region and task_s
        if (t == 0) {
            const unsigned int q = atomicAdd(a.status + 1, 1u);
            int ok = 1;
            if (q < n_tasks) {
                const int32_t j = (int32_t)(q / (unsigned int)a.R);
                const int32_t r = (int32_t)(q % (unsigned int)a.R);
                if (j > 0) {
                    unsigned int seen = 0;
                    for (unsigned long long it = 0; it < kHandoffSpinLimit; ++it) {
                        seen = ld_acquire_gpu(a.handoff_flag + r);
                        if (seen >= (unsigned int)j) break;
                        __nanosleep(256);
                    }
                    if (seen < (unsigned int)j) {
                        atomicOr(a.status, 1u);
                        ok = 0;
                    }
                }
            }
            task_s[slot][0] = q < n_tasks ? (int)q : -1;
            task_s[slot][1] = ok;
        }
        named_bar(bar_id, a.tpr);
        const int q = task_s[slot][0];
        if (q < 0) break;
        if (!task_s[slot][1]) continue;   // the wait gave up: skip this chunk (status set)
        const int32_t j = q / a.R, r = q % a.R;
        const int32_t s0 = j * K, s1 = min(a.S, s0 + K);
        uint8_t* region = a.handoff + (size_t)r * (size_t)a.handoff_bytes;
        if (j > 0) __threadfence();
        replica_body<F, Z, RULE, KIND>(a, slot, t, r, base, s0, s1, j > 0 ? region : nullptr,
                                       s1 < a.S ? region : nullptr);
        if (s1 < a.S) {
            __threadfence();
            named_bar(bar_id, a.tpr);
            if (t == 0) st_release_gpu(a.handoff_flag + r, (unsigned int)(j + 1));
        }
    }
}

// Many instances in one persistent launch: every thread group repeatedly claims
// the next (instance, replica) unit from a global counter (units are ordered by
// decreasing cost on the host) and runs it with that instance's arguments,
// copied into shared memory.
template <class F, class Z, int RULE, int KIND, bool SMEM>
__global__ void __launch_bounds__(512, 1) batch_kernel(const BatchArgs b) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    __shared__ SweepArgs args_s[15];
    __shared__ int unit_s[15];
    const int slot = threadIdx.x / b.tpr;
    const int t = threadIdx.x - slot * b.tpr;
    if (slot >= b.rpc) return;
    const int bar_id = 1 + slot;
    uint8_t* base = SMEM ? (smem_raw + (size_t)slot * (size_t)b.slot_bytes)
                         : (b.gstate + ((size_t)blockIdx.x * b.rpc + slot) * (size_t)b.slot_bytes);
    for (;;) {
        if (t == 0) unit_s[slot] = (int)atomicAdd(b.counter, 1u);
        named_bar(bar_id, b.tpr);
        const int u = unit_s[slot];
        if (u >= b.n_units) break;
        const BatchUnit un = b.units[u];
        const uint32_t* src = reinterpret_cast<const uint32_t*>(b.insts + un.inst);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&args_s[slot]);
        for (int w = t; w < (int)(sizeof(SweepArgs) / 4); w += b.tpr) dst[w] = src[w];
        named_bar(bar_id, b.tpr);
        replica_body<F, Z, RULE, KIND>(args_s[slot], slot, t, un.replica, base);
        named_bar(bar_id, b.tpr);   // the group is done with args_s and unit_s
    }
}

}  // namespace dev
}  // namespace sa
