/*
 * mars.h: C ABI of the GB300 (sm_103a) MARS library.
 *
 * MARS, "Mean-field Annealing from a Random State" (Yavorsky, Markovich,
 * Polyakov, Rubtsov, arXiv 1907.05124), searches for low-energy spin states of
 * the Ising problem of Section 2, Eq. 2:
 *
 *     E(sigma) = sum_{i<j} J_ij sigma_i sigma_j + sum_i h_i sigma_i,
 *
 * with J symmetric, zero diagonal, sigma in {-1,+1}^n. (Eq. 2 sums each pair
 * twice; this library reports every pair once, so Eq. 2's value is
 * 2E - sum_i h_i sigma_i.) Max-cut with weights w is the same problem with
 * J = w; its cut (Eq. 3) is (sum_{i<j} w_ij - E) / 2 when h = 0.
 *
 * The method (Section 3, Algorithm 1) runs many independent replicas. Each
 * starts from s_i ~ U(-1,1) and a start temperature t0 ~ U(t_min, t_max),
 * lowers T by c_step while T stays positive, and at each temperature repeats
 * sweeps  s_i <- -tanh(Phi_i / T),  Phi_i = sum_j J_ij s_j + h_i,  until the
 * largest change d of a sweep is at most d_min (or k_max sweeps were done).
 * The final s is rounded to spins (sign(0) = +1) and the best replica kept.
 *
 * A sweep visits the spins sequentially, each new s_i used at once by the
 * spins after it (Gauss-Seidel: the per-spin update of Section 3). The visiting
 * order is a property of the instance (see mars_instance_csr). The synchronous
 * reading of Algorithm 1's listing is available as MARS_UPDATE_JACOBI.
 *
 * Conventions for every call:
 *  - Return value: MARS_OK (0) or a negative mars_status; the message of the
 *    last failure is available from mars_last_error. The library never aborts
 *    the process.
 *  - Pointers are host pointers unless the call's flags hold MARS_DEVICE_PTR,
 *    in which case they are device pointers on the context's device. Inputs are
 *    read during the call only and copied; the caller keeps ownership of every
 *    buffer it passes.
 *  - Work is ordered on the CUDA stream given to mars_create. Blocking calls
 *    (mars_solve, mars_energy, mars_draw_replicas) synchronise that stream
 *    before they return.
 *  - A context is not thread-safe: serialise calls on one context.
 */
#ifndef MARS_H
#define MARS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mars_ctx mars_ctx;

typedef enum {
    MARS_OK = 0,
    MARS_EINVAL = -1,    /* bad argument: asymmetric J, non-zero diagonal, bad CSR, ... */
    MARS_ENOMEM = -2,    /* device allocation failed or the HBM budget would be exceeded */
    MARS_EAGAIN = -3,    /* result not ready yet (non-blocking calls) */
    MARS_ETIMEOUT = -4,  /* a bounded device-side wait gave up */
    MARS_EDEVICE = -5,   /* a CUDA call failed */
    MARS_ENOTFOUND = -6, /* unknown instance or request id */
    MARS_ECANCELED = -7  /* the request was cancelled (mars_cancel) */
} mars_status;

typedef enum { MARS_I8 = 1, MARS_F32 = 2, MARS_F64 = 3 } mars_dtype;

enum {
    MARS_DEVICE_PTR = 1u,
    /* mars_params.flags: after a MARS_BF16 descent of a dense instance,
     * re-converge every replica's last level with FP32 local fields (the
     * SIMT path), from its BF16 final state at that level's temperature.
     * Its sweeps are added to the replica's counts. */
    MARS_POLISH_FP32 = 2u
};

typedef enum { MARS_UPDATE_GS = 0, MARS_UPDATE_JACOBI = 1 } mars_update;

typedef enum {
    MARS_FP32 = 0,  /* local fields in FP32 (the parity path) */
    MARS_BF16 = 1,  /* dense J*m with BF16 operands, FP32 accumulation */
    MARS_FP8 = 2    /* dense J*m with E4M3 operands (integer J only), FP32 accumulation */
} mars_precision;

/*
 * Create a context on CUDA device `device`. hbm_budget_bytes caps the device
 * memory the context holds at any time (0 = no cap). cuda_stream is a
 * cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream) or NULL for a
 * stream the context creates and owns.
 */
int mars_create(mars_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream);

/* Release every instance and buffer of the context. NULL is ignored. */
void mars_destroy(mars_ctx* ctx);

/* Message of the last failed call on this context (never NULL). */
const char* mars_last_error(mars_ctx* ctx);

/*
 * Register a dense instance (Section 2, Eq. 2). J is n*n row-major of type jt
 * (MARS_I8, MARS_F32 or MARS_F64) and must be exactly symmetric with a zero
 * diagonal; h (n doubles, host) may be NULL for h = 0. order (n int32, host,
 * nullable) is the sweep's spin visiting order, a permutation of 0..n-1;
 * NULL means 0..n-1. On success *inst receives the instance id.
 * Errors: MARS_EINVAL (n <= 0, asymmetric J, non-zero diagonal, non-finite
 * value, order not a permutation), MARS_ENOMEM, MARS_EDEVICE.
 */
int mars_instance_dense(mars_ctx* ctx, int32_t n, const void* J, int32_t jt, const double* h,
                        const int32_t* order, uint32_t flags, int32_t* inst);

/*
 * Register a sparse instance in CSR form: row_ptr (n+1 int32, row_ptr[0] = 0,
 * non-decreasing, row_ptr[n] = nnz), col (nnz int32 in [0, n), no repeated
 * column in a row, no diagonal entry), val (nnz of type vt). Both directions
 * of every coupling must be present with the same value. h (n doubles, host)
 * may be NULL. order (n int32, host) is the sweep's visiting order; NULL asks
 * the library for a greedy colouring order (colour classes in turn, index
 * order within a class; mars_instance_order returns it). Any order gives the
 * same result as a strictly sequential sweep in that order: spins whose
 * earlier-visited neighbours are all settled are updated together.
 * Errors: MARS_EINVAL (bad CSR, asymmetry, diagonal, order), MARS_ENOMEM,
 * MARS_EDEVICE.
 */
int mars_instance_csr(mars_ctx* ctx, int32_t n, int64_t nnz, const int32_t* row_ptr,
                      const int32_t* col, const void* val, int32_t vt, const double* h,
                      const int32_t* order, uint32_t flags, int32_t* inst);

/* Release an instance's device data. Errors: MARS_ENOTFOUND. */
int mars_instance_free(mars_ctx* ctx, int32_t inst);

typedef struct {
    int32_t n;
    int32_t dense;           /* 1 for a dense instance, 0 for CSR */
    int64_t nnz;             /* stored off-diagonal couplings (both directions) */
    int32_t levels;          /* parallel steps of one sweep (colour classes for a colour order) */
    int32_t integer;         /* 1 if every J_ij and h_i is an integer: energies are exact int64 */
    double total_weight;     /* sum_{i<j} J_ij, for cut = (total_weight - E) / 2 */
    int64_t device_bytes;    /* device memory held by the instance */
} mars_instance_info;

/* Describe an instance. Errors: MARS_ENOTFOUND. */
int mars_instance_get_info(mars_ctx* ctx, int32_t inst, mars_instance_info* info);

/* Copy the instance's sweep order (n int32, host) into order_out. */
int mars_instance_order(mars_ctx* ctx, int32_t inst, int32_t* order_out);

/*
 * Parameters of one solve (Section 3, Algorithm 1; the paper uses c_step = 1
 * and d_min = 1e-4 for every experiment, Section 4.1).
 *  replicas      number of independent descents R (>= 1)
 *  t_min, t_max  start temperatures are drawn uniformly from [t_min, t_max]
 *  c_step        temperature decrement per level (> 0); t_max / c_step and every
 *                t0 / c_step must be at most 1e6 (levels per replica)
 *  d_min         a level ends when the sweep's largest |change| is <= d_min
 *  k_max         cap on sweeps per level (>= 1); capped levels are counted
 *  fixed_sweeps  > 0: exactly this many sweeps per level instead of the rule
 *  seed, stream  counter-based start-state draw: Philox4x32-10 with key
 *                (seed low word, seed high word); s_i of replica r is
 *                2u-1 with u = (word (i mod 4) of Philox(i/4, r, 0, stream) >> 8) 2^-24;
 *                t0_r = float(t_min + u (t_max - t_min)) with u from word 0 of
 *                Philox(0, r, 1, stream), in double without fused operations
 *  update        MARS_UPDATE_GS (default) or MARS_UPDATE_JACOBI
 *  precision     mars_precision of the local-field product
 *  m0, t0        optional caller start states: m0 R*n floats (replica-major,
 *                original spin labels, values in [-1, 1]) and t0 R floats;
 *                NULL draws them as above
 *  flags         MARS_DEVICE_PTR if m0/t0 are device pointers; MARS_POLISH_FP32
 *  schedule      MARS_SCHEDULE_LINEAR (default, the paper's: T <- T - c_step
 *                while T > 0) or MARS_SCHEDULE_GEOMETRIC (a labelled variant:
 *                T <- cool_ratio T while T > t_floor, 0 < cool_ratio < 1,
 *                t_floor > 0, at most 1e6 levels)
 *  quench        nonzero: after the last level, one more level at the T -> 0+
 *                limit of the update, s_i <- -sgn(Phi_i) (0 for a zero
 *                field), until no spin changes or k_max sweeps (a labelled
 *                variant: Algorithm 1's last decrement taken to T = 0); it
 *                counts as a level and ignores fixed_sweeps
 *  method        MARS_METHOD_MARS (default: Algorithm 1) or MARS_METHOD_NMFA,
 *                noisy mean-field annealing as Section 2 surveys it: every
 *                iteration computes, synchronously for all spins,
 *                Phi_i = (h_i + sum_j J_ij s_j) / sqrt(h_i^2 + sum_j J_ij^2)
 *                + nmfa_sigma xi_i and shat_i = -tanh(Phi_i / T), then sets
 *                s_i <- nmfa_alpha shat_i + (1 - nmfa_alpha) s_i and lowers T
 *                by the schedule: one iteration per level (update, d_min,
 *                k_max and fixed_sweeps are not used; quench is refused).
 *                xi_i ~ N(0, 1) is counter-based: Philox (key = seed words)
 *                at counter (i/2, r, 2 + k, stream) gives words w0, w1 for
 *                replica r, iteration k (from 0 over all levels), original
 *                spin label i; u1 = ((w0 >> 8) + 1) 2^-24, u2 = (w1 >> 8)
 *                2^-24 and the Box-Muller transform gives sqrt(-2 ln u1)
 *                cos(2 pi u2) for even i, sqrt(-2 ln u1) sin(2 pi u2) for odd
 *                i. A spin without coupling or field has Phi_i = sigma xi_i.
 *                FP32 precision only; dense and CSR instances.
 *  nmfa_alpha    mixing weight in [0, 1] (NMFA)
 *  nmfa_sigma    noise standard deviation >= 0 (NMFA)
 */
typedef enum { MARS_SCHEDULE_LINEAR = 0, MARS_SCHEDULE_GEOMETRIC = 1 } mars_schedule;
typedef enum { MARS_METHOD_MARS = 0, MARS_METHOD_NMFA = 1 } mars_method;
typedef struct {
    int32_t replicas;
    double t_min, t_max, c_step, d_min;
    int32_t k_max;
    int32_t fixed_sweeps;
    uint64_t seed;
    uint32_t stream;
    int32_t update;
    int32_t precision;
    const float* m0;
    const float* t0;
    uint32_t flags;
    int32_t schedule;
    double cool_ratio, t_floor;
    int32_t quench;
    int32_t method;
    double nmfa_alpha, nmfa_sigma;
} mars_params;

/* Fill p with the paper's defaults: c_step 1, d_min 1e-4, k_max 1000, GS, FP32,
 * method MARS (nmfa_alpha 0.5, nmfa_sigma 0). */
void mars_params_default(mars_params* p);

/*
 * Optional per-replica outputs of a solve. Every pointer may be NULL. With
 * MARS_DEVICE_PTR in flags they are device pointers, else host pointers.
 *  energies  R doubles       exact energy of each replica's spins
 *  spins     R*n int8        each replica's sign-rounded spins (original labels)
 *  m_final   R*n float       each replica's final magnetisation (original labels)
 *  t0        R float         the start temperatures used
 *  sweeps    R int32         sweeps done;  levels: R int32 levels visited;
 *  capped    R int32         levels ended by k_max
 */
typedef struct {
    double* energies;
    int8_t* spins;
    float* m_final;
    float* t0;
    int32_t* sweeps;
    int32_t* levels;
    int32_t* capped;
    uint32_t flags;
} mars_outputs;

typedef struct {
    double best_energy;       /* E of the best replica (exact; see energy_err_bound) */
    int64_t best_energy_i64;  /* the same as an integer when the instance is integer */
    double best_cut;          /* (total_weight - best_energy) / 2: the max-cut value when h = 0 */
    int32_t best_replica;     /* lowest replica index among those with the best energy */
    int32_t hits;             /* replicas whose energy equals the best */
    double mean_energy;       /* mean energy over replicas */
    int64_t sweeps;           /* sweeps over all replicas */
    int64_t spin_updates;     /* sum over sweeps of n (one s_i per spin per sweep) */
    int64_t levels;           /* temperature levels over all replicas */
    int64_t capped_levels;    /* levels ended by k_max */
    double gpu_seconds;       /* device time of the solve (CUDA events) */
    double descent_seconds;   /* device time of the descent alone: start states to final
                                 magnetisations, without the energies and the argmin */
    double energy_err_bound;  /* 0 when energies are exact */
    int32_t status;           /* MARS_OK or the device-side error */
    int32_t integer;          /* 1 if energies are exact integers */
    /* Tensor-core path only (precision BF16): CUDA-event time, count and
     * algorithmic flops (2 x 128 x n per active replica) of the panel GEMM
     * launches of one sampled sweep per batch of sweeps; 0 elsewhere. */
    double gemm_seconds;
    int64_t gemm_launches;
    double gemm_flops;
    /* Kernels launched for this result (a captured sweep's graph nodes
     * counted one by one); mars_solve_batch reports the whole batch's count
     * in every job's result; 0 from the serving calls. */
    int64_t kernel_launches;
    /* Level-synchronous sparse path only (magnetisations in global memory,
     * mars_solve): CUDA-event time, count and spin-updates (live replicas x
     * spins of the level) of the level launches of one sampled sweep per
     * batch of sweeps; 0 elsewhere. */
    double level_seconds;
    int64_t level_launches;
    int64_t level_updates;
} mars_result;

/*
 * Run MARS on an instance and block until done. best_spins (n int8, host,
 * nullable) receives the best replica's spins in the caller's labels.
 * outputs and result may be NULL. Errors: MARS_EINVAL (bad parameters),
 * MARS_ENOTFOUND, MARS_ENOMEM, MARS_ETIMEOUT, MARS_EDEVICE.
 */
int mars_solve(mars_ctx* ctx, int32_t inst, const mars_params* params, int8_t* best_spins,
               const mars_outputs* outputs, mars_result* result);

/*
 * Several solves in one persistent launch (the batch of Section 3's
 * independent simulations, across instances). Job j solves CSR instance
 * insts[j] with params[j] (sequential FP32 sweeps); results[j] and, when
 * best_spins and best_spins[j] are non-NULL, best_spins[j] (n_j int8, host)
 * receive what mars_solve would return: every replica's result is the same
 * as in a separate mars_solve with the same parameters. Instances of uneven
 * size and replica count share the SMs: CTAs drain one instance's replica
 * queue after another. gpu_seconds and descent_seconds of every result time
 * the whole batch. Errors: as mars_solve, plus MARS_EINVAL for a dense
 * instance or one too large for the on-chip kernel.
 */
int mars_solve_batch(mars_ctx* ctx, int32_t count, const int32_t* insts, const mars_params* params,
                     int8_t* const* best_spins, mars_result* results);

/*
 * Launch shape of an instance's solves. The paper has no counterpart: these
 * knobs choose how the same arithmetic is laid out on the GPU. -1 leaves a
 * knob to the library's default (or to its MARS_* environment override).
 *   sell_rt          sparse sliced-ELL kernel: replica slots per CTA, 1|2|4
 *   sell_threads     threads per CTA, 512|1024
 *   sell_smem_table  couplings staged in shared memory when they fit, 0|1
 *   tc_rpw           dense BF16 tensor-core descent: replicas per chain warp, 1|2|4
 *   tc_overlap       panel p+1's GEMM overlapped with panel p's chain, 0|1
 *   tc_pair          panels 2q and 2q+1 share one GEMM (one pass over the
 *                    magnetisations per pair of panels), 0|1; with tc_pair
 *                    the overlap is off
 * tc_overlap and tc_pair change results only by rounding: the previous
 * panel's part of a panel's fields is then summed in FP32 instead of through
 * the low-precision GEMM.
 */
typedef struct mars_shape {
    int32_t sell_rt, sell_threads, sell_smem_table;
    int32_t tc_rpw, tc_overlap, tc_pair;
} mars_shape;

/* Set (shape non-NULL) or clear (NULL) an instance's launch shape.
 * Errors: MARS_ENOTFOUND, MARS_EINVAL for a value outside the sets above. */
int mars_set_shape(mars_ctx* ctx, int32_t inst, const mars_shape* shape);
int mars_get_shape(mars_ctx* ctx, int32_t inst, mars_shape* out);

/*
 * Autotuner for batched execution (the launch shape is not in the paper).
 * Times every candidate shape of the path that params select (sparse
 * sliced-ELL: slots x threads x table placement; dense BF16: replicas per
 * warp x overlap) on `repeats` blocking solves with params each, keeps the
 * fastest descent, stores that shape on the instance for later solves and
 * returns it in *best (nullable) with its time in *seconds (nullable). A
 * path with no choices times the default once per repeat. Blocking; the
 * caller's params drive every trial, so tune on a short schedule (e.g.
 * fixed_sweeps) when a full solve is long. Errors: as mars_solve, plus
 * MARS_EINVAL for repeats outside [1, 100]; on error the previous shape
 * stays.
 */
int mars_autotune(mars_ctx* ctx, int32_t inst, const mars_params* params, int32_t repeats,
                  mars_shape* best, double* seconds);

/*
 * Serving. Requests are solves queued with mars_submit and collected with
 * mars_poll; each mars_submit / mars_poll call advances the engine. Queued
 * requests are admitted in arrival order whenever an in-flight slot is free
 * (mars_serve_limits, default 8) and the context's HBM budget holds the
 * request's buffers; each admitted request runs on its own CUDA stream, so
 * requests that arrive while others are on the GPU start as soon as slots
 * and memory free up and their kernels overlap on the device. Sparse
 * requests run on persistent CTAs that stay resident while work lasts; they
 * hold at most half of the SMs (MARS_SERVE_SPARSE_SMS, read when the engine
 * starts, sets another count), so dense requests' kernels always find SMs
 * free. A request's
 * result is the same as mars_solve's with the same parameters, except that
 * replicas run in index order (the per-replica results are identical).
 * m0/t0 must be device pointers (MARS_DEVICE_PTR) or NULL; the instance must
 * stay registered until the request is collected.
 */
int mars_serve_limits(mars_ctx* ctx, int32_t max_inflight);

/* Queue a solve; *req receives its id. Errors: as mars_solve's parameter checks. */
int mars_submit(mars_ctx* ctx, int32_t inst, const mars_params* params, int64_t* req);

/*
 * MARS_OK with the request's best spins (n int8, host, nullable) and result
 * (nullable) once it is done (the request is then forgotten); MARS_EAGAIN
 * while it is queued or running; the request's error if it failed;
 * MARS_ENOTFOUND for an unknown id.
 */
int mars_poll(mars_ctx* ctx, int64_t req, int8_t* best_spins, mars_result* result);

/*
 * Cancel a request. A queued request is dropped at once; a running one keeps
 * its kernels in flight (a dense tensor-core request stops after its current
 * batch of sweeps), its results are discarded and its buffers freed when they
 * end. Either way the request's mars_poll returns MARS_ECANCELED once.
 * Errors: MARS_ENOTFOUND for an unknown (or already collected) id.
 */
int mars_cancel(mars_ctx* ctx, int64_t req);

/* Numbers of queued and running requests (after advancing the engine). */
int mars_serve_status(mars_ctx* ctx, int32_t* queued, int32_t* running);

/*
 * Requests served so far by route: ring_jobs ran as jobs of the persistent
 * serving kernel (sparse instances with integer couplings whose state fits
 * on chip: each is published into a device-side ring that the running
 * kernel's CTAs take work from, so a request that arrives while others run
 * joins the same launch); stream_jobs ran their own kernels on their own
 * stream (dense requests and the rest). Either pointer may be NULL.
 */
int mars_serve_counters(mars_ctx* ctx, int64_t* ring_jobs, int64_t* stream_jobs);

/*
 * Failure detection: a device-side bounded wait on a host-mapped flag, the
 * signalling the serving engine's results travel by. One thread of a kernel
 * polls the flag for at most budget_us microseconds (by its own clock64);
 * the host raises the flag right after the launch. MARS_OK when the kernel
 * saw the flag in time; MARS_ETIMEOUT when the wait gave up (the kernel
 * records that in a status word and exits; the context stays usable);
 * MARS_EINVAL for budget_us outside [1, 10^7]. The paper has no counterpart
 * (it is part of the serving engine's failure detection).
 *
 * Host-side fault injection for tests reads the environment variable
 * MARS_FAULT when the context is created: a comma-separated list of
 *   alloc:K  the K-th device allocation of the context fails (MARS_ENOMEM)
 *   flag     mars_device_check never raises its flag (its wait runs out)
 */
int mars_device_check(mars_ctx* ctx, int32_t budget_us);

/*
 * Exact energies (Section 2, Eq. 2, pairs once) of count spin vectors
 * (count*n int8, entries +-1, caller labels). e (count doubles) receives the
 * energy rounded once to the nearest double; e_i64 (nullable) receives it as
 * an integer for integer instances. spins/e/e_i64 follow flags. Errors:
 * MARS_EINVAL (an entry not +-1), MARS_ENOTFOUND, MARS_EDEVICE.
 */
int mars_energy(mars_ctx* ctx, int32_t inst, const int8_t* spins, int32_t count, double* e,
                int64_t* e_i64, uint32_t flags);

/*
 * The start-state draw alone (see mars_params): replicas r0 .. r0+R-1 with n
 * spins. m0 (R*n floats) and t0 (R floats) follow flags; either may be NULL.
 */
int mars_draw_replicas(mars_ctx* ctx, uint64_t seed, uint32_t stream, int32_t r0, int32_t R,
                       int32_t n, double t_min, double t_max, float* m0, float* t0,
                       uint32_t flags);

/*
 * Bytes of the static device array behind mars_solve_noalloc (16 MiB).
 */
#define MARS_NOALLOC_SCRATCH_BYTES (16u << 20)

/*
 * mars_solve_noalloc: the solve of mars_solve without allocating any device
 * memory. The paper has no counterpart to this entry point. It is for
 * callers that cannot allocate device memory while they run: a program whose
 * device memory is already reserved in full by another framework's allocator,
 * or a latency-bound loop that must not call an allocator (or handle its
 * failure) once it has started. Such a caller registers its instances at
 * start-up, when allocation is still allowed, and solves them with this call.
 *
 * Every per-solve buffer (start temperatures, the replica queue, per-replica
 * spins and energies, counters, the result) lives in one file-scope static
 * device array of MARS_NOALLOC_SCRATCH_BYTES. Each GPU that loads the library
 * holds that array until the process exits. The call allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.
 *  - Inputs: an instance registered earlier, and params as for mars_solve
 *    with update MARS_UPDATE_GS, precision MARS_FP32 and t0 = NULL (the
 *    start temperatures are always drawn); m0 may be a device pointer
 *    (MARS_DEVICE_PTR) or NULL.
 *  - Outputs: best_spins (n int8, device pointer, required), energies
 *    (R doubles, device pointer, or NULL) and result (host, or NULL). Replicas
 *    run in index order instead of longest-first; each replica's result is
 *    the same as mars_solve's for the same seed.
 *  - Limit: the replica count and n must fit the array (about R*n + 40*R
 *    bytes); larger requests, and instances too large for the on-chip kernels,
 *    return MARS_EINVAL with a message naming the limit.
 *  - Set-up: the first call with a context looks up the array's device
 *    address with cudaGetSymbolAddress (with the context's device current)
 *    and caches it in the context; make that first call before any stream
 *    capture on the device. The device must not be reset while the context
 *    lives (a reset invalidates the cached address along with the context's
 *    own buffers): after a reset, destroy the context and create a new one.
 *  - Sharing: all calls share the one array and each starts by clearing the
 *    counters it needs at zero. Calls whose work overlaps on the GPU (other
 *    streams, other contexts, other threads) race on the array: serialise
 *    them.
 */
int mars_solve_noalloc(mars_ctx* ctx, int32_t inst, const mars_params* params, int8_t* best_spins,
                       double* energies, mars_result* result);

#ifdef __cplusplus
}
#endif
#endif
