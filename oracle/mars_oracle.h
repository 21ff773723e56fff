/*
 * MARS oracle: a plain, slow, FP64 CPU restatement of the method of
 * "Highly parallel algorithm for the Ising ground state searching problem"
 * (Yavorsky, Markovich, Polyakov, Rubtsov; arXiv 1907.05124).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links or calls
 * this code; only the tests, the package's smoke entry and the benchmark's
 * CPU-baseline leg do. It shares no code with the CUDA path.
 *
 * Problem (Section 2, Eq. 2): spins sigma in {-1,+1}^n, symmetric couplings J
 * with a zero diagonal, field h. The reported energy counts every pair once:
 *     E(sigma) = sum_{i<j} J_ij sigma_i sigma_j + sum_i h_i sigma_i
 * (Eq. 2 sums each pair twice; with h = 0 that is 2E). The max-cut value of
 * Eq. 3 with weights w = J is cut = (sum_{i<j} w_ij - E_pair) / 2.
 *
 * Method (Section 3, Algorithm 1): every replica starts from s_i ~ U(-1,1) and
 * a start temperature t; it lowers T by C_step while T stays positive and at
 * each level repeats sweeps s_i <- -tanh(Phi_i / T), Phi_i = sum_j J_ij s_j
 * + h_i, until the largest change d of a sweep is at most d_min.
 */
#ifndef MARS_ORACLE_H
#define MARS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Couplings: dense row-major J (n*n) when J != NULL, else CSR. h may be NULL. */
typedef struct {
    int32_t n;
    const double* J;
    const int32_t* row_ptr;
    const int32_t* col;
    const double* val;
    const double* h;
} or_instance;

typedef struct {
    int64_t sweeps;         /* sweeps done over all levels */
    int64_t levels;         /* temperature levels visited (T > 0) */
    int64_t capped_levels;  /* levels ended by k_max while d > d_min */
    double final_T;         /* temperature of the last level visited, 0 if none */
    double last_d;          /* d of the last sweep, 0 if none */
} or_replica_stats;

enum { OR_UPDATE_GS = 0, OR_UPDATE_JACOBI = 1 };

/*
 * Cooling schedule. NULL (or all zero) is the paper's Algorithm 1: T <- T -
 * C_step before each level, levels while T > 0. The rest are labelled
 * variants, not the paper's schedule:
 *   geometric: T <- ratio * T before each level (0 < ratio < 1), levels
 *              while T > t_floor (> 0);
 *   quench:    after the last level, one more level at the T -> 0+ limit of
 *              the update, s_i <- -sgn(Phi_i) with 0 for Phi_i = 0 (Algorithm
 *              1's last decrement taken to T = 0), sweeps until no spin
 *              changes (d = 0 <= d_min) or k_max; it counts as a level.
 */
typedef struct {
    int32_t geometric;
    double ratio;
    double t_floor;
    int32_t quench;
} or_schedule;

/* Phi_i = sum_{j != i} J_ij s_j + h_i, summed in column order, then h added. */
double or_local_field(const or_instance* in, const double* s, int32_t i);

/*
 * One replica of Algorithm 1. m holds s on entry (the start state) and the
 * final s on return. order is the sweep's spin order (NULL = 0..n-1).
 * fixed_sweeps > 0 replaces the stopping rule by exactly that many sweeps per
 * level (the quench level keeps its own rule). update selects sequential (GS)
 * or synchronous (Jacobi) sweeps. scratch: n doubles, needed for Jacobi only.
 * sch: the cooling schedule (NULL = the paper's). Returns 0, or -1 on bad
 * input.
 */
int or_mars_replica(const or_instance* in, const int32_t* order, double* m, double t0,
                    double c_step, double d_min, int32_t k_max, int32_t fixed_sweeps,
                    int32_t update, double* scratch, const or_schedule* sch, or_replica_stats* st);

/*
 * R replicas with start states m0 (R*n floats, replica-major) and start
 * temperatures t0 (R floats). Outputs are optional (NULL to skip): final m
 * (R*n doubles), sign-rounded spins (R*n, sign(0) = +1), exact energies (R),
 * stats (R). nthreads > 1 runs replicas on that many OpenMP threads when the
 * library was built with OpenMP. Returns 0, or -1 on bad input.
 */
int or_mars_solve(const or_instance* in, const int32_t* order, int32_t R, const float* m0,
                  const float* t0, double c_step, double d_min, int32_t k_max,
                  int32_t fixed_sweeps, int32_t update, const or_schedule* sch, int32_t nthreads,
                  double* m_out, int8_t* sigma_out, double* energy_out, or_replica_stats* stats_out);

/* Exact energy of spins (entries +-1), rounded once to the nearest double. */
double or_energy(const or_instance* in, const int8_t* sigma);
/* The same energy written as (1/2) sigma^T J sigma + h.sigma in plain doubles. */
double or_energy_quadratic(const or_instance* in, const int8_t* sigma);
/* Cut weight: exact sum of w_ij over pairs i<j with sigma_i != sigma_j. */
double or_cut(const or_instance* in, const int8_t* sigma);
/* Exactly rounded sum of count doubles (the accumulator behind the two above). */
double or_exact_sum(const double* x, int64_t count);

/*
 * Ground state by Gray-code enumeration of all 2^n states (n <= 30). Returns
 * the minimum energy (exact), one minimising configuration and the number of
 * minimising states (|E - E_min| <= tol). Returns 0, or -1 on bad input.
 */
int or_bruteforce(const or_instance* in, double tol, double* e_min, int8_t* sigma_min,
                  int64_t* n_min);

/*
 * Noisy mean-field annealing (NMFA), the alternative method the paper surveys
 * in Section 2 (its "normalised mean-field terms plus Gaussian noise" and the
 * convex combination). One iteration computes, for every spin from the same
 * state s (synchronously),
 *     Phi_i  = (h_i + sum_{j != i} J_ij s_j) / sqrt(h_i^2 + sum_{j != i} J_ij^2) + sigma xi_i,
 *     shat_i = -tanh(Phi_i / T),
 * then sets s_i <- alpha shat_i + (1 - alpha) s_i for every i and lowers T
 * by the schedule: one iteration per temperature level, levels while T > 0
 * (or T > t_floor when geometric; the quench flag is not used). A spin with
 * no coupling and no field has Phi_i = sigma xi_i. xi_i ~ N(0, 1) is drawn by
 * or_nmfa_normal for (replica r, iteration k counted from 0 over all levels,
 * spin i). Replica stats count one sweep per level; capped_levels is 0.
 */

/*
 * The standard normal of NMFA's noise, restated from its definition: Philox
 * with key (seed low word, seed high word) at counter (i/2, r, 2 + k, stream)
 * gives words w0, w1; u1 = ((w0 >> 8) + 1) 2^-24 in (0, 1], u2 = (w1 >> 8)
 * 2^-24; the Box-Muller transform (Box and Muller, 1958) gives
 * sqrt(-2 ln u1) cos(2 pi u2) for even i and sqrt(-2 ln u1) sin(2 pi u2) for
 * odd i, in double.
 */
double or_nmfa_normal(uint64_t seed, uint32_t stream, uint32_t r, uint32_t k, uint32_t i);

int or_nmfa_replica(const or_instance* in, double* m, double t0, double c_step, double alpha,
                    double sigma, uint64_t seed, uint32_t stream, uint32_t r, double* scratch,
                    const or_schedule* sch, or_replica_stats* st);

/* R replicas of NMFA; replica q uses noise index r = q and the outputs of
 * or_mars_solve. scratch is internal. Returns 0, or -1 on bad input. */
int or_nmfa_solve(const or_instance* in, int32_t R, const float* m0, const float* t0, double c_step,
                  double alpha, double sigma, uint64_t seed, uint32_t stream, const or_schedule* sch,
                  int32_t nthreads, double* m_out, int8_t* sigma_out, double* energy_out,
                  or_replica_stats* stats_out);

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/*
 * The library's counter-based draw of start states, restated from its
 * definition: key = (seed low word, seed high word);
 * m0[r][i] = 2u - 1 with u = (word (i mod 4) of Philox(ctr = (i/4, r, 0, stream)) >> 8) * 2^-24;
 * t0[r] = float(t_min + u (t_max - t_min)) with u from word 0 of
 * Philox(ctr = (0, r, 1, stream)), evaluated in double without fused operations.
 * Writes replicas r0 .. r0+R-1 into m0 (R*n) and t0 (R).
 */
void or_draw_replicas(uint64_t seed, uint32_t stream, int32_t r0, int32_t R, int32_t n,
                      double t_min, double t_max, float* m0, float* t0);

#ifdef __cplusplus
}
#endif
#endif
