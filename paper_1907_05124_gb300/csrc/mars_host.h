// Host-side internals shared by the runtime's translation units: the context,
// registered instances, device allocation under the HBM budget, error
// reporting, and the entry points between the solve orchestration
// (mars_api.cu), the tensor-core descent driver (mars_tc_driver.cu) and the
// serving engine (mars_serve.cu).
#pragma once

#include "../../include/mars.h"
#include "mars_internal.h"

#include <cudaTypedefs.h>

#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

using namespace mars;

// Upper bound on temperature levels per replica (t0 / c_step), so that every
// descent ends and T - c_step always lowers T in double precision.
constexpr double kMaxLevels = 1e6;

// Levels a replica with start temperature t0 visits under p's schedule (an
// upper bound, counting a quench level).
double levels_bound(const mars_params* p, double t0);

// The labelled schedule variants' parameters; the paper's linear schedule
// needs none.
bool schedule_ok(const mars_params* p);

// Why p's method settings are refused (null when they are fine), and the
// method's settings of a descent: NMFA runs synchronous sweeps, one per level.
const char* method_error(const mars_params* p);
void set_method(DevSolve& s, const mars_params* p);

template <class S>
void set_schedule(S& s, const mars_params* p)
{
    s.geometric = p->schedule == MARS_SCHEDULE_GEOMETRIC ? 1 : 0;
    s.cool_ratio = p->cool_ratio;
    s.t_floor = p->t_floor;
    s.quench = p->quench ? 1 : 0;
}


struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Instance {
    DevInstance dev;
    std::vector<int32_t> order;     // caller's visiting order (new label a visits order[a]... see build)
    std::vector<DevMem> mem;
    mars_instance_info info{};
    double abs_weight = 0.0;        // sum_{i<j} |J_ij| + sum |h_i| (error bound of float energies)
};


struct Serve;  // the serving engine's request table (mars_serve.cu)
void serve_release(mars_ctx* c);
void serve_delete(Serve* sv);

struct mars_ctx {
    std::unique_ptr<Serve, void (*)(Serve*)> serve{nullptr, nullptr};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0;
    size_t used = 0;
    int sms = 0;
    std::string err = "no error";
    std::map<int32_t, std::unique_ptr<Instance>> insts;
    int32_t next_id = 1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;  // ev3: end of the descent
    std::vector<cudaEvent_t> prof;  // event pairs around sampled panel GEMM launches
    void* noalloc_base = nullptr;   // device address of mars_solve_noalloc's static array
    // host-side fault injection (MARS_FAULT, read at creation): the
    // allocation that fails (1-based count, 0 = none) and a withheld flag
    int64_t fault_alloc_at = 0, allocs = 0;
    bool fault_flag = false;
    // mars_device_check: host-mapped flag and its device status word
    int32_t* check_flag = nullptr;
    int32_t* check_status = nullptr;
    ~mars_ctx()
    {
        for (cudaEvent_t e : prof) cudaEventDestroy(e);
    }
};

// Records the message for mars_last_error and returns code.
int fail(mars_ctx* c, int code, const char* fmt, ...);

#define MARS_CUDA(c, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((c), MARS_EDEVICE, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Device memory under the context's HBM budget (stream-ordered).
int dev_alloc(mars_ctx* c, size_t bytes, DevMem* out);
int dev_alloc_on(mars_ctx* c, size_t bytes, DevMem* out, cudaStream_t st);
void dev_free_on(mars_ctx* c, DevMem* m, cudaStream_t st);
void dev_free(mars_ctx* c, DevMem* m);

// RAII set of device buffers freed at scope exit (stream-ordered).
struct Scratch {
    mars_ctx* c;
    std::vector<DevMem> bufs;
    explicit Scratch(mars_ctx* ctx) : c(ctx) {}
    ~Scratch()
    {
        for (auto& b : bufs) dev_free(c, &b);
    }
    template <typename T>
    int get(size_t count, T** out)
    {
        DevMem m;
        int rc = dev_alloc(c, count * sizeof(T), &m);
        if (rc) return rc;
        bufs.push_back(m);
        *out = (T*)m.p;
        return MARS_OK;
    }
};

Instance* find(mars_ctx* c, int32_t id);

// Reads MARS_FAULT's items into the context (mars_device_check documents them).
void parse_faults(mars_ctx* c, const char* spec);

// Value of an integer environment override, or dflt.
int env_flag(const char* name, int dflt);

// The dense descent on tensor cores: slots in start-temperature order, a
// sweep = for each 128-spin panel {BF16 panel GEMM, in-panel sequential
// chain}, then the level step; the host checks the active count between
// batches of sweeps. Writes the same per-replica outputs as the other paths.
struct TcProfile {
    double gemm_seconds = 0.0, gemm_flops = 0.0;
    int64_t gemm_launches = 0;
    int64_t launches = 0;  // every kernel of the descent, graph nodes counted one by one
};

// One dense tensor-core descent in flight: its device state, tensor maps and
// the host's view of progress. run_dense_tc drives it to the end; the serving
// engine steps it one batch of sweeps at a time.
struct TcRun {
    TcState t;
    TcPanel g;
    CUtensorMap tmJ, tmS;
    int P = 0, ntiles = 0, splitk = 1, batch = 1;
    int64_t done_sweeps = 0, sweep_cap = 0;
    int32_t* h_counters = nullptr;  // pinned: active prefix, active count, error
    int32_t active_at_batch = 0;
    bool profile = false;
    // One sweep (128-spin panels x {GEMM, chain}, then the level step) captured
    // as a CUDA graph and replayed: 2P+2 launches become one graph launch.
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // Replicas per warp in the chain, and the overlap of panel p+1's GEMM
    // with panel p's chain: the GEMMs run on `side`, the chains on the run's
    // stream, ordered by the events ev (fork, then per panel GEMM done and
    // chain done). G and the chains' next-panel fields Gx alternate between
    // two buffers by panel parity.
    int rpw = 1;
    int chain_warps = 8;               // warps per chain CTA (8, or 4 with few replicas active)
    bool overlap = false;
    bool pair = false;                 // panels 2q, 2q+1 share one GEMM
    std::vector<int> timed_rows;       // rows of each GEMM the profiled sweep timed
    cudaStream_t side = nullptr;
    std::vector<cudaEvent_t> ev;
    float* Gbuf[2] = {nullptr, nullptr};
    float* Gx[2] = {nullptr, nullptr};
    size_t g_floats_max = 0;           // one G buffer at the largest split
    // The plan follows the active replicas from batch to batch unless the
    // instance's shape or an environment override fixes it; chain_slots and
    // gemm_tiles cover the active prefix the plan was made for.
    bool adaptive = false;
    int fixed_rpw = -1, fixed_overlap = -1, fixed_pair = -1;
    int chain_slots = 0, gemm_tiles = 0;
    int sms = 0, kblocks_total = 0;
    // Persistent batches (tc_sweeps_kernel) for a partly active solve: the
    // launch's shape and its counters (2 x kMaxBatch x P + 1 words).
    bool persist = false;
    bool allow_persist = false;        // blocking solves only (not served requests)
    // Between batches the active replicas move to the first slots, so that
    // the plan (GEMM tiles, chain CTAs) covers only them: blocking solves,
    // whose scratch `cp` the solve allocates; rep_mut is t.rep's buffer.
    bool compact = false;
    TcCompact cp;
    int32_t* rep_mut = nullptr;
    int64_t compactions = 0;
    TcPersist pp;
    int32_t* flags = nullptr;
    ~TcRun()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (side) cudaStreamDestroy(side);
    }
};

// Replicas per GEMM tile of the tensor-core path (the MMA's N).
constexpr int kTcBN = 128;
// Most sweeps one batch (one graph replay series or one persistent launch) runs.
constexpr int kTcMaxBatch = 32;

// Allocator the tensor-core set-up draws its buffers from.
using TcGet = std::function<int(size_t, void**)>;

// The tensor-core descent (mars_tc_driver.cu): set-up, one batch of sweeps,
// the host's decision after a batch (1 more, 0 done, < 0 error), and the
// blocking descent of mars_solve.
int tc_setup(mars_ctx* c, const DevInstance& d, const DevSolve& s, const int32_t* rep_dev,
             float t0_max, bool fp8, cudaStream_t st, const TcGet& get, TcRun* run);
int tc_enqueue_batch(mars_ctx* c, TcRun* run, cudaStream_t st);
int tc_after_batch(mars_ctx* c, TcRun* run);
int run_dense_tc(mars_ctx* c, Instance* in, const mars_params* p, const DevSolve& s,
                 const std::vector<int32_t>& reps, float t0_max, Scratch& S, TcProfile* prof,
                 bool polish);

// The level-synchronous sparse descent (mars_wide_driver.cu), blocking: every
// replica resident, a sweep = one launch per level and one decision launch,
// batches of sweeps replayed from a graph until no replica is live; then the
// per-replica outputs. Adds its kernel launches to *launches.
// The first sweep of every batch runs outside the graph with CUDA events
// around each level launch; prof sums their time, count and spin-updates.
struct LevelProfile {
    double seconds = 0.0;
    int64_t launches = 0, updates = 0;
};
int run_sparse_wide(mars_ctx* c, const DevInstance& d, const mars_params* p, const DevSolve& s,
                    const WidePlan& wp, float t0_max, Scratch& S, int64_t* launches, LevelProfile* prof);

// Round-to-nearest-even FP32 -> BF16 bits (host side, for uploads).
uint16_t float_to_bf16_bits(float f);

// The serving engine's progress step (mars_serve.cu).
void serve_progress(mars_ctx* c);
