/*
 * sa_oracle.c -- plain, slow, obviously-correct CPU reference for direct
 * simulated annealing (SA) on QUIO/HUIO problems (K. Suzuki, "Simulated
 * Annealing for Quadratic and Higher-Order Unconstrained Integer
 * Optimization", arXiv:2511.17245).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; it has its own Philox.
 *
 * What it does, in the paper's order:
 *   - merges terms with equal index multisets (Sect. 2, Eqs. def_QUIO/def_HUIO)
 *   - E(z) by direct evaluation of every term (Eq. def_HUIO)
 *   - dE for a candidate value by evaluating the variable's terms at z and at
 *     z' (Eq. energy_diff_quad / energy_diff_poly, first line: the definition
 *     E(z + dz_k) - E(z)); no cached coefficients anywhere
 *   - the SA loop of Sect. 3.1 with sequential visit order and the geometric
 *     schedule T_i
 *   - Metropolis (Sect. 3.3.1), heat bath with the explicit O(u-l) inverse CDF
 *     (Eq. prob_heatbath), optimal-transition Metropolis (Eq. eq_opt_trans) with
 *     a brute-force argmin
 *   - initial/final temperatures of Sect. 3.4 (Eq. eq_temp_init, a = 1/2, b = 0.001)
 *   - exact transition rows and Boltzmann weights for brute-force checks.
 *
 * Integers are exact (int64 results, __int128 intermediates); floating-point
 * models use double.  Where a float decides an integer (accept / reject, the
 * heat-bath pick) the decision is taken in fp32 as the kernel takes it, except
 * that the heat-bath CDF is accumulated in double.  Readings of points the
 * paper leaves open are listed where they are used.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OM_OK 0
#define OM_ERR_INVALID 1
#define OM_ERR_OVERFLOW 2

enum { OM_I32 = 0, OM_I64 = 1, OM_F32 = 2, OM_F64 = 3 };
enum { OM_METROPOLIS = 0, OM_HEAT_BATH = 1, OM_OPT_METROPOLIS = 2 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,   */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11: ten rounds of the   */
/* 4x32 bijection, key bumped by the two Weyl constants between rounds.      */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void om_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Random-number conventions (the paper fixes no generator):
 *   counter = (k, s, r, instance), key = (lo32(seed), hi32(seed)); the
 *   initial state uses s = 0xFFFFFFFF.  One block of 4 words per attempt. */
static void draw_block(uint64_t seed, uint32_t k, uint32_t s, uint32_t r, uint32_t inst,
                       uint32_t out[4])
{
    uint32_t ctr[4] = {k, s, r, inst};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    om_philox4x32_10(ctr, key, out);
}

/* U in [0,1) with 24 random bits; Uc in (0,1]; pick in [0, M). */
static float unit_open_right(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }
static float unit_open_left(uint32_t x) { return (float)((x >> 8) + 1u) * 0x1p-24f; }
static uint32_t pick_below(uint32_t x, uint32_t m) { return (uint32_t)(((uint64_t)x * (uint64_t)m) >> 32); }

/* ------------------------------------------------------------------------ */
/* Model: merged terms + per-variable incidence (plain arrays).              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n;
    int64_t *lo, *hi;
    int32_t n_terms;          /* merged, non-zero, non-constant terms */
    int64_t *t_off;           /* n_terms + 1 */
    int32_t *t_var;           /* sorted multiset per term */
    int is_float;
    int64_t *ci;              /* integer coefficients */
    double *cf;               /* float coefficients */
    int64_t const_i;          /* empty multiset */
    double const_f;
    int64_t *inc_off;         /* n + 1: terms containing variable k */
    int32_t *inc_term;
} om_model;

typedef struct {
    const int32_t *vars;
    int32_t len;
    int64_t ci;
    double cf;
} raw_term;

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int cmp_raw_term(const void *a, const void *b)
{
    const raw_term *p = (const raw_term *)a, *q = (const raw_term *)b;
    if (p->len != q->len) return (p->len > q->len) - (p->len < q->len);
    for (int32_t i = 0; i < p->len; ++i)
        if (p->vars[i] != q->vars[i]) return (p->vars[i] > q->vars[i]) - (p->vars[i] < q->vars[i]);
    return 0;
}

void om_model_destroy(om_model *m)
{
    if (!m) return;
    free(m->lo); free(m->hi); free(m->t_off); free(m->t_var);
    free(m->ci); free(m->cf); free(m->inc_off); free(m->inc_term);
    free(m);
}

/* Builds the merged model.  Readings: duplicate multisets are summed (Sect. 2);
 * terms whose merged coefficient is exactly zero are dropped; the empty multiset
 * is a constant added to E. */
int om_model_create(om_model **out, int32_t n, const int64_t *lo, const int64_t *hi,
                    int64_t n_terms, const int64_t *t_off, const int32_t *t_var,
                    const void *coeffs, int coef_type)
{
    *out = NULL;
    if (n <= 0 || n_terms < 0 || coef_type < 0 || coef_type > 3) return OM_ERR_INVALID;
    for (int32_t i = 0; i < n; ++i)
        if (lo[i] > hi[i]) return OM_ERR_INVALID;
    if (t_off[0] != 0) return OM_ERR_INVALID;
    for (int64_t t = 0; t < n_terms; ++t)
        if (t_off[t + 1] < t_off[t]) return OM_ERR_INVALID;
    for (int64_t j = 0; j < t_off[n_terms]; ++j)
        if (t_var[j] < 0 || t_var[j] >= n) return OM_ERR_INVALID;

    om_model *m = (om_model *)calloc(1, sizeof(om_model));
    m->n = n;
    m->is_float = (coef_type == OM_F32 || coef_type == OM_F64);
    m->lo = (int64_t *)malloc(sizeof(int64_t) * n);
    m->hi = (int64_t *)malloc(sizeof(int64_t) * n);
    memcpy(m->lo, lo, sizeof(int64_t) * n);
    memcpy(m->hi, hi, sizeof(int64_t) * n);

    /* sorted copy of every term's multiset */
    int64_t total = t_off[n_terms];
    int32_t *sorted = (int32_t *)malloc(sizeof(int32_t) * (total > 0 ? total : 1));
    memcpy(sorted, t_var, sizeof(int32_t) * total);
    raw_term *rt = (raw_term *)malloc(sizeof(raw_term) * (n_terms > 0 ? n_terms : 1));
    for (int64_t t = 0; t < n_terms; ++t) {
        int32_t len = (int32_t)(t_off[t + 1] - t_off[t]);
        qsort(sorted + t_off[t], (size_t)len, sizeof(int32_t), cmp_i32);
        rt[t].vars = sorted + t_off[t];
        rt[t].len = len;
        rt[t].ci = 0;
        rt[t].cf = 0.0;
        switch (coef_type) {
        case OM_I32: rt[t].ci = ((const int32_t *)coeffs)[t]; break;
        case OM_I64: rt[t].ci = ((const int64_t *)coeffs)[t]; break;
        case OM_F32: rt[t].cf = ((const float *)coeffs)[t]; break;
        default: rt[t].cf = ((const double *)coeffs)[t]; break;
        }
        if (m->is_float && !isfinite(rt[t].cf)) { free(sorted); free(rt); om_model_destroy(m); return OM_ERR_INVALID; }
    }
    qsort(rt, (size_t)n_terms, sizeof(raw_term), cmp_raw_term);

    /* merge equal multisets */
    m->t_off = (int64_t *)malloc(sizeof(int64_t) * (n_terms + 1));
    m->t_var = (int32_t *)malloc(sizeof(int32_t) * (total > 0 ? total : 1));
    m->ci = (int64_t *)malloc(sizeof(int64_t) * (n_terms > 0 ? n_terms : 1));
    m->cf = (double *)malloc(sizeof(double) * (n_terms > 0 ? n_terms : 1));
    int64_t nt = 0, pos = 0;
    m->t_off[0] = 0;
    for (int64_t t = 0; t < n_terms;) {
        int64_t u = t;
        __int128 si = 0;
        double sf = 0.0;
        while (u < n_terms && cmp_raw_term(&rt[t], &rt[u]) == 0) {
            si += rt[u].ci;
            sf += rt[u].cf;
            ++u;
        }
        if (si > INT64_MAX || si < INT64_MIN) { free(sorted); free(rt); om_model_destroy(m); return OM_ERR_OVERFLOW; }
        int zero = m->is_float ? (sf == 0.0) : (si == 0);
        if (rt[t].len == 0) {
            m->const_i += (int64_t)si;
            m->const_f += sf;
        } else if (!zero) {
            memcpy(m->t_var + pos, rt[t].vars, sizeof(int32_t) * rt[t].len);
            pos += rt[t].len;
            m->ci[nt] = (int64_t)si;
            m->cf[nt] = sf;
            ++nt;
            m->t_off[nt] = pos;
        }
        t = u;
    }
    m->n_terms = (int32_t)nt;
    free(sorted);
    free(rt);

    /* incidence: for each variable, the terms that contain it (once per term) */
    m->inc_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t t = 0; t < nt; ++t)
        for (int64_t j = m->t_off[t]; j < m->t_off[t + 1]; ++j)
            if (j == m->t_off[t] || m->t_var[j] != m->t_var[j - 1]) m->inc_off[m->t_var[j] + 1]++;
    for (int32_t k = 0; k < n; ++k) m->inc_off[k + 1] += m->inc_off[k];
    m->inc_term = (int32_t *)malloc(sizeof(int32_t) * (m->inc_off[n] > 0 ? m->inc_off[n] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * n);
    memcpy(fill, m->inc_off, sizeof(int64_t) * n);
    for (int64_t t = 0; t < nt; ++t)
        for (int64_t j = m->t_off[t]; j < m->t_off[t + 1]; ++j)
            if (j == m->t_off[t] || m->t_var[j] != m->t_var[j - 1]) m->inc_term[fill[m->t_var[j]]++] = (int32_t)t;
    free(fill);
    *out = m;
    return OM_OK;
}

int32_t om_model_n_terms(const om_model *m) { return m->n_terms; }
int64_t om_model_flat_len(const om_model *m) { return m->t_off[m->n_terms]; }
int om_model_is_float(const om_model *m) { return m->is_float; }

/* Copy of the merged term list (for tests). */
void om_model_terms(const om_model *m, int64_t *t_off, int32_t *t_var, int64_t *ci, double *cf)
{
    memcpy(t_off, m->t_off, sizeof(int64_t) * (m->n_terms + 1));
    memcpy(t_var, m->t_var, sizeof(int32_t) * m->t_off[m->n_terms]);
    memcpy(ci, m->ci, sizeof(int64_t) * m->n_terms);
    memcpy(cf, m->cf, sizeof(double) * m->n_terms);
}

/* ------------------------------------------------------------------------ */
/* Energy (Eq. def_HUIO) and the naive energy difference (Eq. energy_diff_poly,
 * first line).                                                              */
/* ------------------------------------------------------------------------ */
static __int128 term_product_i(const om_model *m, int64_t t, const int32_t *z, int32_t k, int64_t zk)
{
    __int128 p = 1;
    for (int64_t j = m->t_off[t]; j < m->t_off[t + 1]; ++j) {
        int32_t v = m->t_var[j];
        p *= (v == k) ? zk : z[v];
    }
    return p;
}

static double term_product_f(const om_model *m, int64_t t, const int32_t *z, int32_t k, double zk)
{
    double p = 1.0;
    for (int64_t j = m->t_off[t]; j < m->t_off[t + 1]; ++j) {
        int32_t v = m->t_var[j];
        p *= (v == k) ? zk : (double)z[v];
    }
    return p;
}

int64_t om_energy_i(const om_model *m, const int32_t *z)
{
    __int128 e = m->const_i;
    for (int64_t t = 0; t < m->n_terms; ++t) e += (__int128)m->ci[t] * term_product_i(m, t, z, -1, 0);
    return (int64_t)e;
}

double om_energy_f(const om_model *m, const int32_t *z)
{
    double e = m->const_f;
    for (int64_t t = 0; t < m->n_terms; ++t) e += m->cf[t] * term_product_f(m, t, z, -1, 0.0);
    return e;
}

/* E(z with z_k = v) - E(z), from the terms that contain k only. */
int64_t om_delta_i(const om_model *m, const int32_t *z, int32_t k, int64_t v)
{
    __int128 d = 0;
    for (int64_t a = m->inc_off[k]; a < m->inc_off[k + 1]; ++a) {
        int64_t t = m->inc_term[a];
        d += (__int128)m->ci[t] * (term_product_i(m, t, z, k, v) - term_product_i(m, t, z, k, z[k]));
    }
    return (int64_t)d;
}

double om_delta_f(const om_model *m, const int32_t *z, int32_t k, double v)
{
    double d = 0.0;
    for (int64_t a = m->inc_off[k]; a < m->inc_off[k + 1]; ++a) {
        int64_t t = m->inc_term[a];
        d += m->cf[t] * (term_product_f(m, t, z, k, v) - term_product_f(m, t, z, k, (double)z[k]));
    }
    return d;
}

/* ------------------------------------------------------------------------ */
/* Schedule (Sect. 3.1): T_i = T_max (T_min/T_max)^((i-1)/(N_sweep-1)).      */
/* Reading: sweep s (0-based) runs at T_{s+1}; a single sweep runs at T_max.  */
/* The kernel-side decision uses beta_s = fp32(1 / T_s).                     */
/* OTM ratio r = s/(N_sweep-1) (Sect. 3.3.3), fp32; 0 for a single sweep.   */
/* ------------------------------------------------------------------------ */
void om_schedule(int32_t n_sweeps, double t_max, double t_min, double *temps, float *beta, float *ratio)
{
    for (int32_t s = 0; s < n_sweeps; ++s) {
        double frac = (n_sweeps > 1) ? (double)s / (double)(n_sweeps - 1) : 0.0;
        double t = t_max * pow(t_min / t_max, frac);
        if (temps) temps[s] = t;
        if (beta) beta[s] = (float)(1.0 / t);
        if (ratio) ratio[s] = (n_sweeps > 1) ? (float)s / (float)(n_sweeps - 1) : 0.0f;
    }
}

/* ------------------------------------------------------------------------ */
/* Initial and final temperature (Sect. 3.4).                                */
/* T_init = -dE_max / ln(1/2),  dE_max ~ max_k sum_m a~_k^(m) (u_k - l_k)^m,  */
/* a~ built from |J| and z^max_i = max(|l_i|, |u_i|);                         */
/* T_final = -dE_min / ln(0.001), dE_min ~ the smallest |J| over all terms.   */
/* ------------------------------------------------------------------------ */
void om_auto_temperatures(const om_model *m, double *t_max, double *t_min)
{
    double de_max = 0.0, de_min = INFINITY;
    for (int32_t k = 0; k < m->n; ++k) {
        double acc = 0.0;
        double width = (double)(m->hi[k] - m->lo[k]);
        for (int64_t a = m->inc_off[k]; a < m->inc_off[k + 1]; ++a) {
            int64_t t = m->inc_term[a];
            double absj = m->is_float ? fabs(m->cf[t]) : fabs((double)m->ci[t]);
            int mult = 0;
            double others = 1.0;
            for (int64_t j = m->t_off[t]; j < m->t_off[t + 1]; ++j) {
                int32_t v = m->t_var[j];
                if (v == k) {
                    ++mult;
                } else {
                    double zm = fmax(fabs((double)m->lo[v]), fabs((double)m->hi[v]));
                    others *= zm;
                }
            }
            /* this term contributes |J| prod z^max to a~_k^(mult) times (u_k-l_k)^mult */
            acc += absj * others * pow(width, (double)mult);
        }
        if (acc > de_max) de_max = acc;
    }
    for (int64_t t = 0; t < m->n_terms; ++t) {
        double absj = m->is_float ? fabs(m->cf[t]) : fabs((double)m->ci[t]);
        if (absj > 0 && absj < de_min) de_min = absj;
    }
    if (!isfinite(de_min)) de_min = 1.0;
    if (de_max <= 0.0) de_max = de_min;
    *t_max = -de_max / log(0.5);
    *t_min = -de_min / log(0.001);
}

/* ------------------------------------------------------------------------ */
/* One attempt on variable k.                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t near_threshold;   /* decisions within the margin of the threshold */
    int64_t followed;         /* of those, where the trace's choice was adopted */
    int64_t mismatch;         /* trace disagreed outside every margin          */
    int64_t first_bad_s, first_bad_k, first_bad_r;
    int64_t first_bad_oracle, first_bad_trace;
} om_follow_stats;

typedef struct {
    int rule;
    float beta;
    float ratio;
    double margin;       /* relative near-threshold margin */
} attempt_ctx;

/* dE for candidate value v of variable k (int or float model), as double for
 * float models and exact int64 otherwise. */
static void delta_value(const om_model *m, const int32_t *z, int32_t k, int64_t v, int64_t *di, double *df)
{
    if (m->is_float) *df = om_delta_f(m, z, k, (double)v);
    else *di = om_delta_i(m, z, k, v);
}

static float delta_as_float(const om_model *m, int64_t di, double df)
{
    return m->is_float ? (float)df : (float)di;
}

static int delta_nonpositive(const om_model *m, int64_t di, double df)
{
    return m->is_float ? (df <= 0.0) : (di <= 0);
}

/* Metropolis acceptance (Sect. 3.3.1): accept if dE <= 0 or U < exp(-dE/T),
 * evaluated as U01(x) < expf(-fp32(dE) * beta) in fp32.  Reports how close U is
 * to the threshold so that the caller can treat near-threshold events. */
static int metropolis_accept(const om_model *m, int64_t di, double df, uint32_t xu, float beta,
                             double margin, int *near)
{
    *near = 0;
    if (delta_nonpositive(m, di, df)) return 1;
    float x = delta_as_float(m, di, df) * beta;
    float p = expf(-x);
    float u = unit_open_right(xu);
    if (fabs((double)u - (double)p) <= margin * (double)p) *near = 1;
    return u < p;
}

/* Uniform nonzero change (Sect. 3.3.1): one of the u-l values other than z. */
static int64_t propose_uniform(const om_model *m, const int32_t *z, int32_t k, uint32_t x)
{
    uint32_t width = (uint32_t)(m->hi[k] - m->lo[k]);
    uint32_t off = (uint32_t)(z[k] - m->lo[k]);
    uint32_t j = pick_below(x, width);
    if (j >= off) ++j;
    return m->lo[k] + (int64_t)j;
}

/* Brute-force argmin over v in [l,u], v != z (Eq. eq_opt_trans); ties go to the
 * smallest v.  Reading: "all possible changes" means the nonzero ones. */
static int64_t argmin_change(const om_model *m, const int32_t *z, int32_t k)
{
    int64_t best_v = 0;
    int have = 0;
    int64_t best_i = 0;
    double best_f = 0.0;
    for (int64_t v = m->lo[k]; v <= m->hi[k]; ++v) {
        if (v == z[k]) continue;
        int64_t di = 0;
        double df = 0.0;
        delta_value(m, z, k, v, &di, &df);
        int better = !have || (m->is_float ? (df < best_f) : (di < best_i));
        if (better) {
            best_v = v;
            best_i = di;
            best_f = df;
            have = 1;
        }
    }
    return best_v;
}

/* Heat bath (Eq. prob_heatbath) with the explicit inverse CDF over every value
 * in [l,u] (current value included, dE = 0 there).  Weights are
 * expf(-fp32(dE_v - dE_min) * beta) (the shift by the minimum is for range and
 * does not change the distribution); the CDF is accumulated in double; the pick
 * is the smallest v with C_v >= Uc * C_total, Uc in (0,1].
 * When `want` is a value in range, reports whether picking it instead is
 * consistent with the CDF within the margin. */
static int64_t heat_bath_pick(const om_model *m, const int32_t *z, int32_t k, uint32_t x, float beta,
                              double margin, int64_t want, int *near, int *want_ok)
{
    int64_t lo = m->lo[k], hi = m->hi[k];
    int64_t n = hi - lo + 1;
    int64_t *di = (int64_t *)malloc(sizeof(int64_t) * n);
    double *df = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) {
        di[i] = 0;
        df[i] = 0.0;
        if (lo + i != z[k]) delta_value(m, z, k, lo + i, &di[i], &df[i]);
    }
    int64_t min_i = di[0];
    double min_f = df[0];
    for (int64_t i = 1; i < n; ++i) {
        if (di[i] < min_i) min_i = di[i];
        if (df[i] < min_f) min_f = df[i];
    }
    double total = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        float gap = m->is_float ? (float)(df[i] - min_f) : (float)(di[i] - min_i);
        w[i] = (double)expf(-(gap * beta));
        total += w[i];
    }
    double thr = (double)unit_open_left(x) * total;
    double cum = 0.0;
    int64_t pick = n - 1;
    for (int64_t i = 0; i < n; ++i) {
        cum += w[i];
        if (cum >= thr) { pick = i; break; }
    }
    /* boundary check: C_{pick-1} < thr <= C_pick */
    double c_hi = 0.0;
    for (int64_t i = 0; i <= pick; ++i) c_hi += w[i];
    double c_lo = c_hi - w[pick];
    *near = (fabs(thr - c_hi) <= margin * total) || (pick > 0 && fabs(thr - c_lo) <= margin * total);
    if (want_ok) {
        *want_ok = 0;
        if (want >= lo && want <= hi) {
            int64_t wi = want - lo;
            double a = 0.0;
            for (int64_t i = 0; i < wi; ++i) a += w[i];
            double b = a + w[wi];
            /* want is valid iff C_{want-1} - eps <= thr <= C_want + eps */
            if (thr >= a - margin * total && thr <= b + margin * total) *want_ok = 1;
        }
    }
    free(di); free(df); free(w);
    return lo + pick;
}

/* One attempt; returns the value after the attempt.  `want` < INT64_MIN+1
 * disables following.  Counts near-threshold events and mismatches. */
typedef struct {
    int64_t new_v;
    int changed;
    int64_t de_i;
    double de_f;
} attempt_out;

static attempt_out attempt(const om_model *m, const int32_t *z, int32_t k, uint64_t seed, uint32_t s,
                           uint32_t r, uint32_t inst, const attempt_ctx *cx, int follow, int64_t want,
                           om_follow_stats *st)
{
    attempt_out res = {z[k], 0, 0, 0.0};
    uint32_t x[4];
    if (m->hi[k] == m->lo[k]) return res;          /* fixed variable: skipped */
    draw_block(seed, (uint32_t)k, s, r, inst, x);
    int64_t v = z[k];
    int near = 0;
    if (cx->rule == OM_HEAT_BATH) {
        int want_ok = 0;
        v = heat_bath_pick(m, z, k, x[0], cx->beta, cx->margin, follow ? want : INT64_MIN, &near,
                           follow ? &want_ok : NULL);
        if (near) st->near_threshold++;
        if (follow && want != v) {
            if (want_ok) { st->followed++; v = want; }
            else if (st->mismatch++ == 0) {
                st->first_bad_s = s; st->first_bad_k = k; st->first_bad_r = r;
                st->first_bad_oracle = v; st->first_bad_trace = want;
            }
        }
    } else {
        int64_t prop;
        if (cx->rule == OM_OPT_METROPOLIS && unit_open_right(x[2]) < cx->ratio)
            prop = argmin_change(m, z, k);
        else
            prop = propose_uniform(m, z, k, x[0]);
        int64_t di = 0;
        double df = 0.0;
        delta_value(m, z, k, prop, &di, &df);
        int acc = metropolis_accept(m, di, df, x[1], cx->beta, cx->margin, &near);
        if (near) st->near_threshold++;
        v = acc ? prop : z[k];
        if (follow && want != v) {
            /* only the accept/reject decision may legitimately differ */
            if (near && (want == prop || want == z[k])) { st->followed++; v = want; }
            else if (st->mismatch++ == 0) {
                st->first_bad_s = s; st->first_bad_k = k; st->first_bad_r = r;
                st->first_bad_oracle = v; st->first_bad_trace = want;
            }
        }
    }
    if (v != z[k]) {
        res.changed = 1;
        if (m->is_float) res.de_f = om_delta_f(m, z, k, (double)v);
        else res.de_i = om_delta_i(m, z, k, v);
    }
    res.new_v = v;
    return res;
}

/* ------------------------------------------------------------------------ */
/* The SA run of Sect. 3.1 for replicas [r_begin, r_end).                     */
/*   init z uniformly at random in [l_k, u_k] (reading of "at random");      */
/*   for s = 0..S-1: for k = 0..N-1 in index order: one attempt.             */
/* Optional follow trace: int32 [S][trace_replicas][N] of the values another */
/* implementation held after each attempt; used for replicas < trace_replicas */
/* (indexed by absolute replica number).  trace_out (optional) receives this  */
/* run's own values in the layout [S][r_end - r_begin][N].                    */
/* Outputs per replica (indexed from r_begin): final z [R x N], tracked E,   */
/* recomputed E, number of changes.  Optional best state (best_z, R x N):    */
/* among the states after sweeps 0..S-1 the first with the lowest tracked E  */
/* (the paper is silent on it; it names the optimal solution as the goal,    */
/* Sect. 2), with its recomputed E in best_e_i / best_e_f.                   */
/* ------------------------------------------------------------------------ */
int om_run(const om_model *m, int rule, int32_t n_sweeps, uint64_t seed, uint32_t inst,
           double t_max, double t_min, double margin,
           int32_t r_begin, int32_t r_end, const int32_t *init_states,
           const int32_t *trace, int32_t trace_replicas,
           int32_t *out_z, int64_t *out_e_i, double *out_e_f,
           int64_t *out_e_recomputed_i, double *out_e_recomputed_f,
           int64_t *out_changes, om_follow_stats *stats,
           int64_t *energy_trace_i, double *energy_trace_f, int32_t *trace_out,
           int32_t *best_z, int64_t *best_e_i, double *best_e_f)
{
    if (rule < 0 || rule > 2 || n_sweeps < 1 || r_end < r_begin) return OM_ERR_INVALID;
    int32_t n = m->n;
    double *temps = (double *)malloc(sizeof(double) * n_sweeps);
    float *beta = (float *)malloc(sizeof(float) * n_sweeps);
    float *ratio = (float *)malloc(sizeof(float) * n_sweeps);
    om_schedule(n_sweeps, t_max, t_min, temps, beta, ratio);
    om_follow_stats st;
    memset(&st, 0, sizeof(st));
    st.first_bad_s = st.first_bad_k = st.first_bad_r = -1;

    for (int32_t r = r_begin; r < r_end; ++r) {
        int32_t *z = out_z + (int64_t)(r - r_begin) * n;
        if (init_states) {
            memcpy(z, init_states + (int64_t)(r - r_begin) * n, sizeof(int32_t) * n);
        } else {
            for (int32_t k = 0; k < n; ++k) {
                uint32_t x[4];
                draw_block(seed, (uint32_t)k, 0xFFFFFFFFu, (uint32_t)r, inst, x);
                uint32_t cnt = (uint32_t)(m->hi[k] - m->lo[k]) + 1u;
                z[k] = (int32_t)(m->lo[k] + (int64_t)pick_below(x[0], cnt));
            }
        }
        int64_t e_i = m->is_float ? 0 : om_energy_i(m, z);
        double e_f = m->is_float ? om_energy_f(m, z) : 0.0;
        int64_t changes = 0;
        int follow = (trace != NULL) && (r < trace_replicas);
        /* best state at sweep ends: strictly lower tracked energy replaces it */
        int have_best = 0;
        int64_t bst_i = 0;
        double bst_f = 0.0;
        int32_t *bz = best_z ? best_z + (int64_t)(r - r_begin) * n : NULL;
        for (int32_t s = 0; s < n_sweeps; ++s) {
            attempt_ctx cx = {rule, beta[s], ratio[s], margin};
            for (int32_t k = 0; k < n; ++k) {
                int64_t want = 0;
                if (follow) want = trace[((int64_t)s * trace_replicas + r) * n + k];
                attempt_out a = attempt(m, z, k, seed, (uint32_t)s, (uint32_t)r, inst, &cx, follow, want, &st);
                if (a.changed) {
                    z[k] = (int32_t)a.new_v;
                    e_i += a.de_i;
                    e_f += a.de_f;
                    ++changes;
                }
                if (trace_out) trace_out[((int64_t)s * (r_end - r_begin) + (r - r_begin)) * n + k] = z[k];
            }
            if (energy_trace_i) energy_trace_i[(int64_t)s * (r_end - r_begin) + (r - r_begin)] = e_i;
            if (energy_trace_f) energy_trace_f[(int64_t)s * (r_end - r_begin) + (r - r_begin)] = e_f;
            if (bz && (!have_best || (m->is_float ? e_f < bst_f : e_i < bst_i))) {
                have_best = 1;
                bst_i = e_i;
                bst_f = e_f;
                memcpy(bz, z, sizeof(int32_t) * n);
            }
        }
        int64_t idx = r - r_begin;
        if (bz && best_e_i) best_e_i[idx] = m->is_float ? 0 : om_energy_i(m, bz);
        if (bz && best_e_f) best_e_f[idx] = m->is_float ? om_energy_f(m, bz) : (double)om_energy_i(m, bz);
        if (out_e_i) out_e_i[idx] = e_i;
        if (out_e_f) out_e_f[idx] = e_f;
        if (out_e_recomputed_i) out_e_recomputed_i[idx] = m->is_float ? 0 : om_energy_i(m, z);
        if (out_e_recomputed_f) out_e_recomputed_f[idx] = m->is_float ? om_energy_f(m, z) : (double)om_energy_i(m, z);
        if (out_changes) out_changes[idx] = changes;
    }
    if (stats) *stats = st;
    free(temps); free(beta); free(ratio);
    return OM_OK;
}

/* Single attempt exposed for distribution tests: given z, variable k and the
 * four counter words, returns the value after the attempt. */
int64_t om_attempt(const om_model *m, const int32_t *z, int32_t k, int rule, float beta, float ratio,
                   uint64_t seed, uint32_t s, uint32_t r, uint32_t inst)
{
    attempt_ctx cx = {rule, beta, ratio, 0.0};
    om_follow_stats st;
    memset(&st, 0, sizeof(st));
    attempt_out a = attempt(m, z, k, seed, s, r, inst, &cx, 0, 0, &st);
    return a.new_v;
}

/* Brute-force argmin exposed for tests. */
int64_t om_argmin_change(const om_model *m, const int32_t *z, int32_t k) { return argmin_change(m, z, k); }

/* ------------------------------------------------------------------------ */
/* Exact transition probabilities of one single-variable update at fixed T,  */
/* in double, straight from the rules' definitions (Sect. 3.3):               */
/*   Metropolis: P(v) = min(1, e^{-dE_v/T}) / (u-l) for v != z              */
/*   heat bath : P(v) = e^{-dE_v/T} / sum_j e^{-dE_j/T}                     */
/*   OTM       : two-stage proposal (prob r: argmin, else uniform nonzero)  */
/*               with Metropolis acceptance                                  */
/* out[i] is the probability of ending at value l+i.                          */
/* ------------------------------------------------------------------------ */
void om_transition_row(const om_model *m, const int32_t *z, int32_t k, int rule, double temp, double ratio,
                       double *out)
{
    int64_t lo = m->lo[k], hi = m->hi[k];
    int64_t n = hi - lo + 1;
    for (int64_t i = 0; i < n; ++i) out[i] = 0.0;
    if (n == 1) { out[0] = 1.0; return; }
    double *de = (double *)malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t di = 0;
        double df = 0.0;
        if (lo + i == z[k]) { de[i] = 0.0; continue; }
        delta_value(m, z, k, lo + i, &di, &df);
        de[i] = m->is_float ? df : (double)di;
    }
    int64_t cur = z[k] - lo;
    if (rule == OM_HEAT_BATH) {
        double mn = de[0];
        for (int64_t i = 1; i < n; ++i) if (de[i] < mn) mn = de[i];
        double tot = 0.0;
        for (int64_t i = 0; i < n; ++i) { out[i] = exp(-(de[i] - mn) / temp); tot += out[i]; }
        for (int64_t i = 0; i < n; ++i) out[i] /= tot;
    } else {
        double q = (rule == OM_OPT_METROPOLIS) ? ratio : 0.0;
        int64_t amin = argmin_change(m, z, k) - lo;
        double stay = 1.0;
        for (int64_t i = 0; i < n; ++i) {
            if (i == cur) continue;
            double acc = de[i] <= 0 ? 1.0 : exp(-de[i] / temp);
            double prop = (1.0 - q) / (double)(n - 1) + ((i == amin) ? q : 0.0);
            out[i] = prop * acc;
            stay -= out[i];
        }
        out[cur] = stay;
    }
    free(de);
}

/* Number of states of a tiny model (0 if above `cap`). */
int64_t om_state_count(const om_model *m, int64_t cap)
{
    int64_t c = 1;
    for (int32_t k = 0; k < m->n; ++k) {
        c *= (m->hi[k] - m->lo[k] + 1);
        if (c > cap) return 0;
    }
    return c;
}

/* Enumerates every state in mixed-radix order (variable 0 fastest) and writes
 * E(z) for each; states_out (optional) receives the states. */
void om_enumerate(const om_model *m, int64_t count, double *energies, int32_t *states_out)
{
    int32_t n = m->n;
    int32_t *z = (int32_t *)malloc(sizeof(int32_t) * n);
    for (int32_t k = 0; k < n; ++k) z[k] = (int32_t)m->lo[k];
    for (int64_t c = 0; c < count; ++c) {
        energies[c] = m->is_float ? om_energy_f(m, z) : (double)om_energy_i(m, z);
        if (states_out) memcpy(states_out + c * n, z, sizeof(int32_t) * n);
        for (int32_t k = 0; k < n; ++k) {
            if (z[k] < m->hi[k]) { z[k]++; break; }
            z[k] = (int32_t)m->lo[k];
        }
    }
    free(z);
}
