// Internal interfaces between the host runtime (mars_api.cu) and the kernels.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mars {

// Device-side status words (status[0]); MARS_OK when clean.
enum DeviceStatus : int32_t { kDevOk = 0, kDevBadIndex = 1, kDevTimeout = 2 };

// Instance data on the device, relabelled so that one sweep is "levels in
// order, any order within a level": new label a has caller label new2old[a].
// Launch-shape choices of an instance's solves, set by mars_autotune or
// mars_set_shape; -1 leaves a knob to its MARS_* environment override, else
// to the built-in default. None changes a replica's arithmetic except
// tc_overlap, which takes the previous panel's part of the fields in FP32.
struct LaunchShape {
    int32_t sell_rt = -1, sell_threads = -1, sell_smem_table = -1;
    int32_t tc_rpw = -1, tc_overlap = -1;
    int32_t tc_pair = -1;  // panel pairs share one GEMM (exclusive with the overlap)
};

struct DevInstance {
    int32_t n = 0;
    int32_t dense = 0;
    int64_t nnz = 0;
    int32_t nlev = 0;
    int32_t integer = 0;
    // sparse (CSR over new labels, columns sorted)
    const int32_t* row_ptr = nullptr;
    const int32_t* col = nullptr;
    const float* val = nullptr;
    const int8_t* val_i8 = nullptr;    // integer instances
    const double* val_f64 = nullptr;   // every instance: exact values for energies
    const int32_t* lvl_start = nullptr;  // nlev+1 offsets into new labels
    // sliced-ELL copy of the couplings: 32-row slices {row0, rows, degree, offset}
    const int4* slices = nullptr;
    const int32_t* lvl_slice = nullptr;  // nlev+1 offsets into slices
    const uint32_t* sell_pm1 = nullptr;  // +-1 couplings: column | sign << 31
    const int2* sell_gen = nullptr;      // general couplings: (column, float bits)
    const uint16_t* sell16 = nullptr;    // +-1 couplings, n < 32768: column | sign << 15
    int32_t nslices = 0;
    int64_t sell_len = 0;                // padded entries (32 x degree summed over slices)
    int32_t regular_deg = 0;             // the common degree when every spin has the same, else 0
    // dense (n*n, new labels: Jn[a][b] = J[new2old[a]][new2old[b]])
    int32_t n_pad = 0;                   // n rounded up to the 128-spin panel
    const __nv_bfloat16* Jbf = nullptr;  // n_pad*n_pad BF16, zero padded (tensor-core operand)
    const float* Jdiag = nullptr;        // (n_pad/128) FP32 128x128 diagonal blocks
    const float* Jsup = nullptr;         // (n_pad/128) FP32 128x128 blocks J[p][p+1] (last: zero)
    const uint8_t* J8 = nullptr;         // n_pad x n_pad E4M3 copy when every J_ij is exact in E4M3
    LaunchShape shape;                   // host-side choice; kernels ignore it
    const float* Jf = nullptr;
    const int8_t* J_i8 = nullptr;
    const double* J_f64 = nullptr;
    // exact FP64 energies of non-integer instances (exact_sum.cuh): every
    // term is a multiple of 2^exact_e0 and every sum fits the accumulator
    int32_t exact_ok = 0;
    int32_t exact_e0 = 0;
    // common
    const float* h = nullptr;          // n floats or null
    const double* h_f64 = nullptr;     // n doubles or null
    const float* inv_norm = nullptr;   // n: 1 / sqrt(h_i^2 + sum_j J_ij^2), 0 where that is 0 (NMFA)
    const int32_t* new2old = nullptr;  // n
};

struct DevResult {
    double best_energy;
    long long best_energy_i64;
    int32_t best_replica;
    int32_t hits;
    double sum_energy;
    long long sweeps;
    long long levels;
    long long capped;
};

// One solve's replica state and outputs (all device pointers).
struct DevSolve {
    int32_t R = 0;
    int32_t ntiles = 0;
    int32_t rt = 1;                    // replicas per tile
    const int32_t* tile_rep = nullptr; // ntiles*rt replica ids (-1 = empty slot)
    const float* t0 = nullptr;         // R start temperatures
    const float* m0 = nullptr;         // R*n caller-labelled start states, or null (draw)
    uint64_t seed = 0;
    uint32_t stream = 0;
    double c_step = 1.0;
    float d_min = 1e-4f;
    int32_t k_max = 1000;
    int32_t fixed_sweeps = 0;
    // labelled schedule variants (schedule.cuh); all zero is the paper's
    int32_t geometric = 0;
    int32_t quench = 0;
    double cool_ratio = 0.5;
    double t_floor = 0.0;
    int32_t jacobi = 0;
    // noisy mean-field annealing (synchronous sweeps, one per level) instead
    // of Algorithm 1's update
    int32_t nmfa = 0;
    float nmfa_alpha = 0.5f, nmfa_sigma = 0.f;
    const double* t_first = nullptr;   // optional per-replica temperature of the first level
    int32_t one_level = 0;             // stop after the first level (the FP32 polish)
    int32_t add_counts = 0;            // add sweeps/levels/capped to the outputs' values
    float* m_scratch = nullptr;        // per-CTA state when it does not fit on chip
    float* m_next = nullptr;           // per-CTA second buffer for synchronous sweeps
    // outputs
    int8_t* sigma = nullptr;           // R*n caller labels
    float* m_final = nullptr;          // R*n caller labels, optional
    double* energy = nullptr;          // R
    long long* energy_i64 = nullptr;   // R
    int32_t* sweeps = nullptr;         // R
    int32_t* levels = nullptr;         // R
    int32_t* capped = nullptr;         // R
    int32_t* work_counter = nullptr;   // 1
    int32_t* status = nullptr;         // 1
    // serving ring only: replicas finished, and a host-mapped flag raised once
    // all R have finished (both null elsewhere)
    int32_t* finished = nullptr;
    int32_t* done_flag = nullptr;
    DevResult* res = nullptr;          // serving ring: the finishing CTA's argmin goes here
    int8_t* best_out = nullptr;        // and the best replica's spins here
};

// One instance of a batched launch (kernels_sparse_sell.cu).
struct BatchJob {
    DevInstance in;
    DevSolve s;
    int32_t fmt = 0;
    int32_t rt = 1;  // replica slots per CTA for this job (1 or 2)
};
// The serving ring: job descriptors the host publishes while the persistent
// serving kernel runs. A job's counters live in the ring (never in request
// buffers), and the host reuses no slot while the kernel lives (it resets the
// ring once the kernel has exited), so a CTA leaving a finished job never
// touches freed memory or another job's counters.
constexpr int kRingCap = 1024;
struct RingSlot {
    int32_t taken = 0;     // replicas taken from the job's queue
    int32_t status = 0;    // device-side error code
    int32_t finished = 0;  // replicas finished
    int32_t pad = 0;
};
struct ServeRing {
    BatchJob jobs[kRingCap];
    RingSlot slots[kRingCap];
    int32_t tail;    // jobs published (job j sits in slot j % kRingCap)
    int32_t cursor;  // first job that may still have replicas to take
    int32_t stop;    // exit once idle
    int32_t pad;
};
// Launch shape of the serving kernel: RT slots, `threads`, dynamic shared
// memory `smem` (the most a job may use) and the grid.
struct RingPlan {
    int rt = 2;
    int threads = 1024;
    size_t smem = 0;
    int grid = 1;
};
bool plan_serve_ring(int device, RingPlan* p);
// Coupling format a job uses under the ring's shared memory (and its slot
// width, 2 when two replicas' magnetisations fit, else 1), or -1 when the
// job's magnetisations do not fit on chip.
int ring_job_format(const DevInstance& in, const RingPlan& p, int* rt);
// Persistent serving kernel: runs published jobs and exits after about
// idle_polls x 2 us without new work (or when ring->stop is set).
cudaError_t launch_serve_ring(ServeRing* ring, const RingPlan& p, int idle_polls, cudaStream_t st);

struct BatchPlan {
    int rt = 1;
    int threads = 1024;
    size_t smem = 0;
    int grid = 0;
};
bool plan_sparse_batch(const DevInstance* ins, int count, int device, BatchPlan* p, int* fmts, int* rts);
cudaError_t launch_sparse_batch(const BatchJob* jobs, int count, int* cursor, const BatchPlan& p,
                                cudaStream_t st);



// Launchers (return cudaError_t of the launch).
struct SparsePlan {
    int rt = 1;         // replicas per tile
    int onchip = 1;     // magnetisations in shared memory (sliced-ELL: else per-CTA slabs)
    int threads = 512;
    size_t smem = 0;    // dynamic shared memory
    int grid = 0;
    size_t scratch_floats = 0;  // m_scratch (+ m_next) floats needed
    int sell = 0;       // the sliced-ELL kernel
    int entry = 0;      // its coupling format: 0 general, 1 +-1 words, 2 +-1 halfwords in smem
    int deg = 0;        // compile-time degree of a regular instance (4 or 6), else 0
};
bool plan_sparse_sell(const DevInstance& in, int R, int device, SparsePlan* p);
// The sliced-ELL kernel with m in global-memory slabs (format 0 or 1, rt 1, 2
// or 4); null for another combination.
const void* pick_sell_slab(int rt, int fmt, int deg);
cudaError_t launch_sparse_sell(const DevInstance& in, const DevSolve& s, const SparsePlan& p,
                               cudaStream_t st);

// Level-synchronous sliced-ELL descent with every replica resident in global
// memory (kernels_sparse_wide.cu): groups of rt slots share one slab layout,
// m[g][i*rt + k]; slot q = g*rt + k runs replica s.tile_rep[q] (-1: empty).
struct DevWide {
    int32_t rt = 4;
    int32_t groups = 0;
    size_t slab = 0;                 // floats per group (sell_slab_floats(n, rt))
    float* m = nullptr;              // groups * slab
    double* T = nullptr;             // per slot: current level's temperature
    float* invT = nullptr;
    int32_t* live = nullptr;         // descending
    int32_t* lvl_sweeps = nullptr;
    int32_t* sweeps = nullptr;
    int32_t* levels = nullptr;
    int32_t* capped = nullptr;
    uint32_t* dmax = nullptr;        // the sweep's largest |change| (float bits, >= 0)
    int32_t* glist = nullptr;        // live groups, ascending
    int32_t* counters = nullptr;     // [0] live groups, [1] live replicas
};
struct WidePlan {
    int rt = 4;
    int entry = 1;      // coupling format: 0 general pairs, 1 +-1 words
    int deg = 0;        // compile-time degree of a regular instance (4 or 6), else 0
    int groups = 0;
    size_t slab = 0;
    int grid = 0;       // CTAs of a level launch
    int sms = 0;
    int staged = 0;     // regular +-1 lattices: neighbour gathers staged in shared memory
    size_t smem = 0;    // the level launch's dynamic shared memory
};
bool plan_sparse_wide(const DevInstance& in, int R, int rt, int device, WidePlan* p);
cudaError_t launch_wide_init(const DevInstance& in, const DevSolve& s, const DevWide& w, const WidePlan& p,
                             cudaStream_t st);
cudaError_t launch_wide_level(const DevInstance& in, const DevSolve& s, const DevWide& w, const WidePlan& p,
                              int level, cudaStream_t st);
// step != 0: the stopping rule and cooling after a sweep; then the live-group
// list and counts (step == 0: the list only).
cudaError_t launch_wide_decide(const DevSolve& s, const DevWide& w, int step, cudaStream_t st);
cudaError_t launch_wide_finalize(const DevInstance& in, const DevSolve& s, const DevWide& w, const WidePlan& p,
                                 cudaStream_t st);
SparsePlan plan_sparse(const DevInstance& in, int R, int jacobi, int device);
cudaError_t launch_sparse(const DevInstance& in, const DevSolve& s, const SparsePlan& p,
                          cudaStream_t st);

// Tensor-core dense path (kernels_dense_tc.cu).
struct TcPanel {
    int32_t p0 = 0;          // first row of the panel
    int32_t kblocks = 0;     // 64-wide K blocks per split
    int32_t R_pad = 0;
    float* G = nullptr;      // [split][R_pad][128]
    float* G1 = nullptr;     // the second panel's partials of a paired GEMM
    int32_t skip_kb = -1;    // first K block of the panel left out (-1: none)
    int32_t fp8 = 0;         // E4M3 operands (K blocks of 128) instead of BF16 (64)
    const int32_t* active_prefix = nullptr;
    int32_t* err = nullptr;
};
struct TcState {
    int32_t R = 0, R_pad = 0, n = 0, n_pad = 0, splitk = 1;
    float* G = nullptr;
    float* S = nullptr;            // [R][n_pad] FP32 magnetisations, slot order
    __nv_bfloat16* Sb = nullptr;   // [R_pad][n_pad] BF16 shadow (tensor-core operand)
    uint8_t* S8 = nullptr;         // [R_pad][n_pad] E4M3 shadow instead, for FP8 descents
    const float* Jdiag = nullptr;
    const float* Jsup = nullptr;       // [P][128][128] FP32 blocks J[p][p+1]
    const float* h = nullptr;
    const int32_t* rep = nullptr;      // slot -> replica
    const int32_t* new2old = nullptr;
    const float* m0 = nullptr;
    const float* t0 = nullptr;
    uint64_t seed = 0;
    uint32_t stream = 0;
    double c_step = 1.0;
    float d_min = 1e-4f;
    int32_t k_max = 1000, fixed_sweeps = 0;
    int32_t geometric = 0, quench = 0;
    double cool_ratio = 0.5, t_floor = 0.0;
    double* T = nullptr;
    float* invT = nullptr;
    float* d = nullptr;
    int32_t* active = nullptr;
    int32_t* levels = nullptr;
    int32_t* lvl_sweeps = nullptr;
    int32_t* sweeps = nullptr;
    int32_t* capped = nullptr;
    int32_t* counters = nullptr;       // [0] active prefix, [1] active count, [2] error
};
// A batch of sweeps in one cooperative launch (tc_sweeps_kernel): n_chain
// chain CTAs, then n_gemm GEMM CTAs, meeting through per-panel counters.
struct TcPersist {
    int32_t n_chain = 0, n_gemm = 0;
    int32_t chain_items = 0;           // replica groups of 8 * rpw slots below the prefix
    int32_t gemm_tiles = 0, splitk = 1;
    int32_t sweeps = 0, P = 0;
    float* G[2] = {nullptr, nullptr};  // split-K partials by panel parity
    float* Gx[2] = {nullptr, nullptr}; // the previous panel's FP32 part of the fields
    int32_t* gemm_done = nullptr;      // [sweeps * P], zero at launch
    int32_t* chain_done = nullptr;     // [sweeps * P], zero at launch
    int32_t* abort = nullptr;          // zero at launch
    long long spin_budget = 0;         // clock64 cycles one wait may take
};
size_t tc_sweeps_smem(int rpw);
cudaError_t launch_tc_sweeps(const CUtensorMap& tmJ, const CUtensorMap& tmS, const TcState& t, const TcPanel& g,
                             const TcPersist& pp, int rpw, cudaStream_t st);
size_t tc_gemm_smem(int bn);
cudaError_t launch_tc_panel_gemm(const CUtensorMap& tmJ, const CUtensorMap& tmS, const TcPanel& g,
                                 int bn, int n_tiles, int splitk, cudaStream_t st);
// Split-K partials a chain with one replica per warp sums; with rpw replicas
// per warp the split must not exceed kChainMaxSplit / rpw.
constexpr int kChainMaxSplit = 16;
// In-panel chain of panel p for rpw (1, 2 or 4) replicas per warp, on the
// split-K fields G; gx_in (nullable) holds the previous panel's FP32 part
// of the fields, and with gx_out (nullable) the chain writes this panel's
// part of the next panel's fields there.
// Panels q and q+1 (first row g.p0) in one pass over K, the second leaving
// panel q's K blocks (from g.skip_kb) out; partials to g.G and g.G1.
cudaError_t launch_tc_pair_gemm(const CUtensorMap& tmJ, const CUtensorMap& tmS, const TcPanel& g, int n_tiles,
                                int splitk, cudaStream_t st);
// cw: warps per chain CTA, 8 or 4 (fewer replica slots per CTA, so a few
// active replicas spread over more SMs); the per-replica arithmetic is the same.
cudaError_t launch_tc_chain(const TcState& t, int p, int rpw, int cw, const float* G, const float* gx_in,
                            float* gx_out, bool g_early, cudaStream_t st);
// Compaction of the active replicas into the first slots: scratch of the
// same shapes as TcState's per-slot arrays (rows of n_pad spins for S and its
// low-precision copy) and the permutation.
struct TcCompact {
    int32_t* perm = nullptr;          // new slot -> old slot, below the prefix
    float* S = nullptr;
    __nv_bfloat16* Sb = nullptr;
    uint8_t* S8 = nullptr;
    double* T = nullptr;
    float* invT = nullptr;
    float* d = nullptr;
    int32_t* active = nullptr;
    int32_t* levels = nullptr;
    int32_t* lvl_sweeps = nullptr;
    int32_t* sweeps = nullptr;
    int32_t* capped = nullptr;
    int32_t* rep = nullptr;
};
// Move the active slots of [0, prefix) to the front, in slot order, and the
// finished ones behind them, in slot order; every per-slot array (magnetisations,
// their low-precision copy, level state, counts, slot -> replica) moves with
// its slot. rep is t.rep's writable buffer. Sets t.counters[0] to the active count.
cudaError_t launch_tc_compact(const TcState& t, int32_t* rep, const TcCompact& cp, int prefix, cudaStream_t st);
cudaError_t launch_tc_init(const TcState& t, cudaStream_t st);
cudaError_t launch_tc_advance(const TcState& t, cudaStream_t st);
cudaError_t launch_tc_prefix(const TcState& t, cudaStream_t st);
cudaError_t launch_tc_finalize(const TcState& t, const DevInstance& in, const DevSolve& s,
                               cudaStream_t st);
// The tensor-core descent's final state in caller labels (R*n floats) and each
// replica's last temperature (0 for a replica that visited no level).
cudaError_t launch_tc_export(const TcState& t, const DevInstance& in, float* m_out, double* t_last,
                             cudaStream_t st);

struct DensePlan {
    int warps_per_block = 4;
    int stages = 0;  // > 0: the staged kernel with this many row buffers
    int onchip = 1;
    size_t smem = 0;
    int grid = 0;
    size_t scratch_floats = 0;
};
DensePlan plan_dense(const DevInstance& in, int R, int jacobi, int device);
cudaError_t launch_dense(const DevInstance& in, const DevSolve& s, const DensePlan& p,
                         cudaStream_t st);

cudaError_t launch_draw(uint64_t seed, uint32_t stream, int32_t r0, int32_t R, int32_t n,
                        double t_min, double t_max, float* m0, float* t0, cudaStream_t st);

cudaError_t launch_queue_identity(int32_t* q, int32_t total, int32_t R, int32_t* counters,
                                  cudaStream_t st);

// One thread polls a host-mapped flag until it is nonzero or budget_cycles of
// its clock64 have passed; then it writes kDevOk or kDevTimeout to *status.
cudaError_t launch_flag_wait(const int32_t* flag, long long budget_cycles, int32_t* status,
                             cudaStream_t st);

cudaError_t launch_best(const DevSolve& s, int32_t n, int32_t integer, int8_t* best_spins,
                        DevResult* res, cudaStream_t st);

cudaError_t launch_energy(const DevInstance& in, const int8_t* spins, int32_t count,
                          double* e, long long* e_i64, int32_t* status, cudaStream_t st);

// Read-only view of a context and one of its instances, for entry points that
// live outside mars_api.cu (mars_noalloc.cu).
struct NoallocView {
    int device = 0;
    cudaStream_t stream = nullptr;
    const DevInstance* inst = nullptr;
    double total_weight = 0.0;
    double energy_err_bound = 0.0;
    void** scratch_base = nullptr;  // the context's cached address of the static array
};

}  // namespace mars

struct mars_ctx;
int noalloc_view(mars_ctx* c, int32_t inst, mars::NoallocView* v);
int noalloc_fail(mars_ctx* c, int code, const char* fmt, ...);
