/*
 * MARS oracle, plain FP64 C. TEST INFRASTRUCTURE ONLY: see mars_oracle.h.
 *
 * Every function restates one definition or one step of the paper:
 *   - energy and cut: Section 2, Eq. 2 (pairs counted once) and Eq. 3;
 *   - the annealing loop: Section 3, Algorithm 1, with the readings listed at
 *     or_mars_replica;
 *   - the start-state draw: the library's documented Philox definition.
 * No blocking, fusion or reordering beyond what those definitions state.
 * Build with -ffp-contract=off so that no multiply-add is fused.
 */
#include "mars_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Exact summation: a wide fixed-point integer, rounded once at the end.     */
/* ------------------------------------------------------------------------ */

/* Value = sum_k d[k] * 2^(32k - ACC_BIAS). 2^-1074 (the smallest double) sits
 * at bit 78 and 2^1024 below bit 2200; 78 limbs leave 2496 bits. */
#define ACC_LIMBS 78
#define ACC_BIAS 1152

typedef struct {
    int64_t d[ACC_LIMBS];
    int64_t pending;
} exact_acc;

static void acc_normalize(exact_acc* a)
{
    int64_t carry = 0;
    for (int k = 0; k < ACC_LIMBS - 1; ++k) {
        int64_t t = a->d[k] + carry;
        a->d[k] = t & 0xffffffffLL;
        carry = (t - a->d[k]) / 4294967296LL; /* exact: t - low is a multiple of 2^32 */
    }
    a->d[ACC_LIMBS - 1] += carry;
    a->pending = 0;
}

static void acc_add(exact_acc* a, double x)
{
    if (x == 0.0) return;
    int e;
    double f = frexp(fabs(x), &e);                 /* |x| = f 2^e, 0.5 <= f < 1 */
    uint64_t mant = (uint64_t)ldexp(f, 53);        /* exact: at most 53 bits */
    int pos = e - 53 + ACC_BIAS;                   /* bit index of mant's unit */
    int k = pos / 32, s = pos % 32;
    unsigned __int128 v = (unsigned __int128)mant << s;
    int64_t c0 = (int64_t)(uint32_t)(v), c1 = (int64_t)(uint32_t)(v >> 32),
            c2 = (int64_t)(uint32_t)(v >> 64);
    if (x < 0) { c0 = -c0; c1 = -c1; c2 = -c2; }
    a->d[k] += c0;
    a->d[k + 1] += c1;
    a->d[k + 2] += c2;
    if (++a->pending >= (1LL << 29)) acc_normalize(a);
}

static int acc_bit(const exact_acc* a, int pos)
{
    if (pos < 0) return 0;
    return (int)((a->d[pos / 32] >> (pos % 32)) & 1);
}

static int acc_any_below(const exact_acc* a, int pos) /* any set bit at index < pos */
{
    for (int p = pos - 1; p >= 0; --p) {
        if ((p % 32) == 31 && a->d[p / 32] == 0) { p -= 31; continue; }
        if (acc_bit(a, p)) return 1;
    }
    return 0;
}

/* Round the exact value to the nearest double, ties to even. */
static double acc_round(exact_acc* a)
{
    acc_normalize(a);
    int neg = a->d[ACC_LIMBS - 1] < 0;
    if (neg) {
        for (int k = 0; k < ACC_LIMBS; ++k) a->d[k] = -a->d[k];
        acc_normalize(a);
    }
    int top = -1;
    for (int p = ACC_LIMBS * 32 - 1; p >= 0; --p) {
        if (acc_bit(a, p)) { top = p; break; }
    }
    if (top < 0) return 0.0;
    int lsb = top - 52;                     /* keep 53 bits ... */
    if (lsb < ACC_BIAS - 1074) lsb = ACC_BIAS - 1074; /* ... or fewer when subnormal */
    uint64_t mant = 0;
    for (int p = top; p >= lsb; --p) mant = (mant << 1) | (uint64_t)acc_bit(a, p);
    int guard = acc_bit(a, lsb - 1);
    int sticky = acc_any_below(a, lsb - 1);
    if (guard && (sticky || (mant & 1))) mant += 1;
    double r = ldexp((double)mant, lsb - ACC_BIAS);
    return neg ? -r : r;
}

double or_exact_sum(const double* x, int64_t count)
{
    exact_acc* a = (exact_acc*)calloc(1, sizeof(exact_acc));
    if (!a) return NAN;
    for (int64_t i = 0; i < count; ++i) acc_add(a, x[i]);
    double r = acc_round(a);
    free(a);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Energy and cut (Section 2, Eq. 2 and Eq. 3)                               */
/* ------------------------------------------------------------------------ */

double or_energy(const or_instance* in, const int8_t* sigma)
{
    exact_acc* a = (exact_acc*)calloc(1, sizeof(exact_acc));
    if (!a) return NAN;
    const int32_t n = in->n;
    for (int32_t i = 0; i < n; ++i) {
        if (in->J) {
            for (int32_t j = i + 1; j < n; ++j)
                acc_add(a, in->J[(int64_t)i * n + j] * (double)(sigma[i] * sigma[j]));
        } else {
            for (int32_t e = in->row_ptr[i]; e < in->row_ptr[i + 1]; ++e) {
                int32_t j = in->col[e];
                if (j > i) acc_add(a, in->val[e] * (double)(sigma[i] * sigma[j]));
            }
        }
        if (in->h) acc_add(a, in->h[i] * (double)sigma[i]);
    }
    double r = acc_round(a);
    free(a);
    return r;
}

double or_energy_quadratic(const or_instance* in, const int8_t* sigma)
{
    double quad = 0.0, lin = 0.0;
    const int32_t n = in->n;
    for (int32_t i = 0; i < n; ++i) {
        double row = 0.0;
        if (in->J) {
            for (int32_t j = 0; j < n; ++j) row += in->J[(int64_t)i * n + j] * sigma[j];
        } else {
            for (int32_t e = in->row_ptr[i]; e < in->row_ptr[i + 1]; ++e)
                row += in->val[e] * sigma[in->col[e]];
        }
        quad += sigma[i] * row;
        if (in->h) lin += in->h[i] * sigma[i];
    }
    return 0.5 * quad + lin;
}

double or_cut(const or_instance* in, const int8_t* sigma)
{
    exact_acc* a = (exact_acc*)calloc(1, sizeof(exact_acc));
    if (!a) return NAN;
    const int32_t n = in->n;
    for (int32_t i = 0; i < n; ++i) {
        if (in->J) {
            for (int32_t j = i + 1; j < n; ++j)
                if (sigma[i] != sigma[j]) acc_add(a, in->J[(int64_t)i * n + j]);
        } else {
            for (int32_t e = in->row_ptr[i]; e < in->row_ptr[i + 1]; ++e) {
                int32_t j = in->col[e];
                if (j > i && sigma[i] != sigma[j]) acc_add(a, in->val[e]);
            }
        }
    }
    double r = acc_round(a);
    free(a);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1                                                               */
/* ------------------------------------------------------------------------ */

double or_local_field(const or_instance* in, const double* s, int32_t i)
{
    double phi = 0.0;
    if (in->J) {
        const double* row = in->J + (int64_t)i * in->n;
        for (int32_t j = 0; j < in->n; ++j)
            if (j != i) phi += row[j] * s[j];
    } else {
        for (int32_t e = in->row_ptr[i]; e < in->row_ptr[i + 1]; ++e)
            if (in->col[e] != i) phi += in->val[e] * s[in->col[e]];
    }
    if (in->h) phi += in->h[i];
    return phi;
}

/*
 * Readings of Algorithm 1 taken here:
 *  - the level loop lowers T by c_step first and visits the level only while
 *    the lowered T is still positive (the text: T decreases to zero);
 *  - "until d > d_min" is read as repeat-until d <= d_min, with k_max as a cap
 *    on the sweeps of one level (the paper states none);
 *  - a GS sweep replaces each s_i as soon as its new value is known, in the
 *    given order (the prose of Section 3 and its per-spin GPU description);
 *    a Jacobi sweep computes every new value from the old vector first;
 *  - Phi_i includes the field h_i (Eq. 2 has it; Algorithm 1 drops it for h=0).
 */
/* -sgn(phi), the update's T -> 0+ limit (0 for phi = 0) */
static double quench_value(double phi) { return phi > 0.0 ? -1.0 : (phi < 0.0 ? 1.0 : 0.0); }

/* One sweep at temperature T (T = 0 selects the quench update); returns d. */
static double sweep(const or_instance* in, const int32_t* order, double* m, double T, int32_t update,
                    double* scratch)
{
    const int32_t n = in->n;
    double d = 0.0;
    if (update == OR_UPDATE_GS) {
        for (int32_t q = 0; q < n; ++q) {
            int32_t i = order ? order[q] : q;
            double phi = or_local_field(in, m, i);
            double shat = T > 0.0 ? -tanh(phi / T) : quench_value(phi);
            double diff = fabs(shat - m[i]);
            if (diff > d) d = diff;
            m[i] = shat;
        }
    } else {
        for (int32_t i = 0; i < n; ++i) {
            double phi = or_local_field(in, m, i);
            scratch[i] = T > 0.0 ? -tanh(phi / T) : quench_value(phi);
            double diff = fabs(scratch[i] - m[i]);
            if (diff > d) d = diff;
        }
        memcpy(m, scratch, sizeof(double) * (size_t)n);
    }
    return d;
}

int or_mars_replica(const or_instance* in, const int32_t* order, double* m, double t0,
                    double c_step, double d_min, int32_t k_max, int32_t fixed_sweeps,
                    int32_t update, double* scratch, const or_schedule* sch, or_replica_stats* st)
{
    if (!in || !m || in->n < 0 || !(c_step > 0) || k_max < 1 || fixed_sweeps < 0) return -1;
    if (update == OR_UPDATE_JACOBI && !scratch) return -1;
    const int geometric = sch && sch->geometric;
    if (geometric && !(sch->ratio > 0.0 && sch->ratio < 1.0 && sch->t_floor > 0.0)) return -1;
    or_replica_stats s = {0, 0, 0, 0.0, 0.0};
    double T = t0;
    for (;;) {
        T = geometric ? T * sch->ratio : T - c_step;
        if (!(T > (geometric ? sch->t_floor : 0.0))) break;
        s.levels += 1;
        s.final_T = T;
        int32_t k = 0;
        double d;
        do {
            d = sweep(in, order, m, T, update, scratch);
            k += 1;
            s.sweeps += 1;
        } while (fixed_sweeps > 0 ? (k < fixed_sweeps) : (d > d_min && k < k_max));
        if (fixed_sweeps == 0 && d > d_min) s.capped_levels += 1;
        s.last_d = d;
    }
    if (sch && sch->quench) {
        s.levels += 1;
        s.final_T = 0.0;
        int32_t k = 0;
        double d;
        do {
            d = sweep(in, order, m, 0.0, update, scratch);
            k += 1;
            s.sweeps += 1;
        } while (d > d_min && k < k_max);
        if (d > d_min) s.capped_levels += 1;
        s.last_d = d;
    }
    if (st) *st = s;
    return 0;
}

int or_mars_solve(const or_instance* in, const int32_t* order, int32_t R, const float* m0,
                  const float* t0, double c_step, double d_min, int32_t k_max,
                  int32_t fixed_sweeps, int32_t update, const or_schedule* sch, int32_t nthreads,
                  double* m_out, int8_t* sigma_out, double* energy_out, or_replica_stats* stats_out)
{
    if (!in || R < 0 || !m0 || !t0) return -1;
    const int32_t n = in->n;
    int bad = 0;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1) reduction(| : bad)
#endif
    for (int32_t r = 0; r < R; ++r) {
        double* m = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 2);
        int8_t* sg = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
        if (!m || !sg) { bad |= 1; free(m); free(sg); continue; }
        for (int32_t i = 0; i < n; ++i) m[i] = (double)m0[(int64_t)r * n + i];
        or_replica_stats st;
        if (or_mars_replica(in, order, m, (double)t0[r], c_step, d_min, k_max, fixed_sweeps,
                            update, m + n, sch, &st) != 0)
            bad |= 1;
        for (int32_t i = 0; i < n; ++i) sg[i] = m[i] >= 0.0 ? 1 : -1;
        if (m_out) memcpy(m_out + (int64_t)r * n, m, sizeof(double) * (size_t)n);
        if (sigma_out) memcpy(sigma_out + (int64_t)r * n, sg, (size_t)n);
        if (energy_out) energy_out[r] = or_energy(in, sg);
        if (stats_out) stats_out[r] = st;
        free(m);
        free(sg);
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Brute force                                                               */
/* ------------------------------------------------------------------------ */

static double coupling(const or_instance* in, int32_t i, int32_t j)
{
    if (in->J) return in->J[(int64_t)i * in->n + j];
    for (int32_t e = in->row_ptr[i]; e < in->row_ptr[i + 1]; ++e)
        if (in->col[e] == j) return in->val[e];
    return 0.0;
}

int or_bruteforce(const or_instance* in, double tol, double* e_min, int8_t* sigma_min,
                  int64_t* n_min)
{
    const int32_t n = in->n;
    if (n < 1 || n > 30) return -1;
    double* Jd = (double*)calloc((size_t)n * n, sizeof(double));
    double* L = (double*)calloc((size_t)n, sizeof(double));
    int8_t* sg = (int8_t*)malloc((size_t)n);
    int8_t* best = (int8_t*)malloc((size_t)n);
    if (!Jd || !L || !sg || !best) { free(Jd); free(L); free(sg); free(best); return -1; }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) Jd[(int64_t)i * n + j] = i == j ? 0.0 : coupling(in, i, j);
    for (int32_t i = 0; i < n; ++i) sg[i] = 1;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) L[i] += Jd[(int64_t)i * n + j];
    double E = or_energy(in, sg);
    double Ebest = E;
    memcpy(best, sg, (size_t)n);
    const uint64_t states = 1ULL << n;
    /* Gray code: state k differs from state k-1 in bit ctz(k). */
    for (uint64_t k = 1; k < states; ++k) {
        int b = __builtin_ctzll(k);
        double hb = in->h ? in->h[b] : 0.0;
        E += -2.0 * sg[b] * (L[b] + hb);
        sg[b] = (int8_t)-sg[b];
        for (int32_t j = 0; j < n; ++j) L[j] += 2.0 * Jd[(int64_t)j * n + b] * sg[b];
        if (E < Ebest) { Ebest = E; memcpy(best, sg, (size_t)n); }
    }
    double exact_best = or_energy(in, best);
    /* Second pass: count states within tol of the minimum (exact energies). */
    int64_t count = 0;
    for (int32_t i = 0; i < n; ++i) sg[i] = 1;
    memset(L, 0, sizeof(double) * (size_t)n);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) L[i] += Jd[(int64_t)i * n + j];
    E = or_energy(in, sg);
    if (fabs(E - exact_best) <= tol + 1e-9 * fabs(exact_best)) count += 1;
    for (uint64_t k = 1; k < states; ++k) {
        int b = __builtin_ctzll(k);
        double hb = in->h ? in->h[b] : 0.0;
        E += -2.0 * sg[b] * (L[b] + hb);
        sg[b] = (int8_t)-sg[b];
        for (int32_t j = 0; j < n; ++j) L[j] += 2.0 * Jd[(int64_t)j * n + b] * sg[b];
        if (fabs(E - exact_best) <= tol + 1e-9 * fabs(exact_best)) count += 1;
    }
    if (e_min) *e_min = exact_best;
    if (sigma_min) memcpy(sigma_min, best, (size_t)n);
    if (n_min) *n_min = count;
    free(Jd); free(L); free(sg); free(best);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 and the start-state draw                                    */
/* ------------------------------------------------------------------------ */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* Round multipliers and key increments from the Philox definition. */
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void or_draw_replicas(uint64_t seed, uint32_t stream, int32_t r0, int32_t R, int32_t n,
                      double t_min, double t_max, float* m0, float* t0)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t q = 0; q < R; ++q) {
        uint32_t r = (uint32_t)(r0 + q);
        uint32_t out[4];
        for (int32_t i = 0; i < n; ++i) {
            if ((i & 3) == 0) {
                const uint32_t ctr[4] = {(uint32_t)i >> 2, r, 0u, stream};
                or_philox4x32_10(ctr, key, out);
            }
            float u = (float)(out[i & 3] >> 8) * 0x1p-24f;
            if (m0) m0[(int64_t)q * n + i] = 2.0f * u - 1.0f;
        }
        const uint32_t ctr_t[4] = {0u, r, 1u, stream};
        or_philox4x32_10(ctr_t, key, out);
        double u = (double)(out[0] >> 8) * 0x1p-24;
        double width = t_max - t_min;
        double prod = u * width;
        double t = t_min + prod;
        if (t0) t0[q] = (float)t;
    }
}

/* ------------------------------------------------------------------------ */
/* Noisy mean-field annealing (Section 2)                                    */
/* ------------------------------------------------------------------------ */

double or_nmfa_normal(uint64_t seed, uint32_t stream, uint32_t r, uint32_t k, uint32_t i)
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {i >> 1, r, 2u + k, stream};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    const double u1 = (double)((w[0] >> 8) + 1u) * 0x1p-24;
    const double u2 = (double)(w[1] >> 8) * 0x1p-24;
    const double rho = sqrt(-2.0 * log(u1));
    const double two_pi = 6.283185307179586476925286766559;
    return (i & 1u) ? rho * sin(two_pi * u2) : rho * cos(two_pi * u2);
}

/* sum_{j != i} J_ij^2 + h_i^2, summed in column order, then h added */
static double field_norm2(const or_instance* in, int32_t i)
{
    double q = 0.0;
    if (in->J) {
        const double* row = in->J + (int64_t)i * in->n;
        for (int32_t j = 0; j < in->n; ++j)
            if (j != i) q += row[j] * row[j];
    } else {
        for (int32_t e = in->row_ptr[i]; e < in->row_ptr[i + 1]; ++e)
            if (in->col[e] != i) q += in->val[e] * in->val[e];
    }
    if (in->h) q += in->h[i] * in->h[i];
    return q;
}

int or_nmfa_replica(const or_instance* in, double* m, double t0, double c_step, double alpha,
                    double sigma, uint64_t seed, uint32_t stream, uint32_t r, double* scratch,
                    const or_schedule* sch, or_replica_stats* st)
{
    if (!in || !m || !scratch || in->n < 0 || !(c_step > 0) || !(alpha >= 0.0 && alpha <= 1.0) ||
        !(sigma >= 0.0))
        return -1;
    const int geometric = sch && sch->geometric;
    if (geometric && !(sch->ratio > 0.0 && sch->ratio < 1.0 && sch->t_floor > 0.0)) return -1;
    const int32_t n = in->n;
    or_replica_stats s = {0, 0, 0, 0.0, 0.0};
    double T = t0;
    uint32_t k = 0;
    for (;;) {
        T = geometric ? T * sch->ratio : T - c_step;
        if (!(T > (geometric ? sch->t_floor : 0.0))) break;
        s.levels += 1;
        s.final_T = T;
        /* every spin's new value from the same state s */
        for (int32_t i = 0; i < n; ++i) {
            const double norm = sqrt(field_norm2(in, i));
            const double field = or_local_field(in, m, i);
            double phi = norm > 0.0 ? field / norm : 0.0;
            if (sigma > 0.0) phi += sigma * or_nmfa_normal(seed, stream, r, k, (uint32_t)i);
            scratch[i] = -tanh(phi / T);
        }
        double d = 0.0;
        for (int32_t i = 0; i < n; ++i) {
            const double v = alpha * scratch[i] + (1.0 - alpha) * m[i];
            const double diff = fabs(v - m[i]);
            if (diff > d) d = diff;
            m[i] = v;
        }
        s.sweeps += 1;
        s.last_d = d;
        k += 1;
    }
    if (st) *st = s;
    return 0;
}

int or_nmfa_solve(const or_instance* in, int32_t R, const float* m0, const float* t0, double c_step,
                  double alpha, double sigma, uint64_t seed, uint32_t stream, const or_schedule* sch,
                  int32_t nthreads, double* m_out, int8_t* sigma_out, double* energy_out,
                  or_replica_stats* stats_out)
{
    if (!in || R < 0 || !m0 || !t0) return -1;
    const int32_t n = in->n;
    int bad = 0;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1) reduction(| : bad)
#endif
    for (int32_t r = 0; r < R; ++r) {
        double* m = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 2);
        int8_t* sg = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
        if (!m || !sg) { bad |= 1; free(m); free(sg); continue; }
        for (int32_t i = 0; i < n; ++i) m[i] = (double)m0[(int64_t)r * n + i];
        or_replica_stats st;
        if (or_nmfa_replica(in, m, (double)t0[r], c_step, alpha, sigma, seed, stream, (uint32_t)r,
                            m + n, sch, &st) != 0)
            bad |= 1;
        for (int32_t i = 0; i < n; ++i) sg[i] = m[i] >= 0.0 ? 1 : -1;
        if (m_out) memcpy(m_out + (int64_t)r * n, m, sizeof(double) * (size_t)n);
        if (sigma_out) memcpy(sigma_out + (int64_t)r * n, sg, (size_t)n);
        if (energy_out) energy_out[r] = or_energy(in, sg);
        if (stats_out) stats_out[r] = st;
        free(m);
        free(sg);
    }
    return bad ? -1 : 0;
}
