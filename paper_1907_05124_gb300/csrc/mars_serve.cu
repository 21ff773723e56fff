// The serving engine behind mars_submit / mars_poll: requests admitted while
// others run (continuous batching), under the HBM budget; sparse integer
// requests become jobs of one persistent serving kernel through a
// device-side job ring, the others run their pipelines on their own streams.
#include "mars_host.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

using namespace mars;

// ---------------------------------------------------------------------------
// Serving: requests admitted while others run (continuous batching).
//
// mars_submit queues a request; every mars_submit / mars_poll call advances
// the engine: finished requests are collected (their events have fired), and
// queued requests are admitted in arrival order while an in-flight slot is
// free and the HBM budget holds their buffers. Each admitted request runs on
// its own stream, so its kernels overlap with the others' on the device; a
// dense tensor-core request advances one batch of sweeps per event.
// ---------------------------------------------------------------------------
enum class ReqState { Queued, Running, TcRunning, RingRunning, Finishing, Done, Failed };

struct ServeReq {
    int64_t id = 0;
    int32_t inst = 0;
    mars_params p{};
    ReqState state = ReqState::Queued;
    int rc = MARS_OK;
    std::string err;
    int slot = -1;
    cudaStream_t st = nullptr;
    std::vector<DevMem> bufs;
    DevSolve s;
    DevInstance dev;
    DevResult* dres = nullptr;
    int8_t* dbest = nullptr;
    unsigned char* pinned = nullptr;  // DevResult | status | counters[4] | best spins
    cudaEvent_t ev = nullptr;
    std::unique_ptr<TcRun> tc;
    double total_weight = 0.0, err_bound = 0.0;
    int64_t ring_job = -1;  // serving-ring job index, or -1
    size_t footprint = 0;   // the admission bound; what the request may allocate
    bool light = false;     // admitted as a serving-ring job (its own in-flight limit)
    bool cancelled = false; // mars_cancel while it ran: discard its results at the end
};

struct Serve {
    std::vector<cudaStream_t> streams;
    std::vector<int> free_slots;
    std::deque<int64_t> queue;
    std::map<int64_t, std::unique_ptr<ServeReq>> reqs;
    int64_t next_id = 1;
    int max_inflight = 8;
    int inflight = 0;
    int light_inflight = 0;  // serving-ring jobs in flight (limit kServeLight)
    // The serving ring: sparse requests run as jobs of one persistent kernel
    // (continuous batching: a job published while the kernel runs is picked
    // up by CTAs as they free up). Descriptors are staged in pinned memory
    // and copied on one publish stream, so the tail the kernel reads never
    // runs ahead of the descriptors it covers.
    bool ring_on = false;
    RingPlan plan;
    ServeRing* ring = nullptr;      // device
    BatchJob* stage_jobs = nullptr; // pinned [kRingCap]
    RingSlot* stage_slots = nullptr;
    int32_t* stage_tail = nullptr;
    int32_t* done = nullptr;        // host-mapped flags [kRingCap]
    int32_t* done_dev = nullptr;
    int ring_refs = 0;              // requests that still read their ring slot
    cudaStream_t pub_st = nullptr, ring_st = nullptr;
    cudaEvent_t ring_ev = nullptr;
    bool kernel_live = false;
    int64_t tail = 0;
    int64_t ring_jobs = 0;          // jobs served through the ring
    int64_t stream_jobs = 0;        // jobs served on their own streams
    int idle_polls = 50;            // about 100 us without work before the kernel exits
    // SMs the persistent serving kernel, and each sparse request on its own
    // stream, may hold at once (MARS_SERVE_SPARSE_SMS, default half the
    // device): their CTAs stay resident while work lasts, and the rest of
    // the device is left to the dense requests' kernels.
    int sparse_sms = 0;
    int sms = 0;
};

// The grid of a persistent sparse launch planned for the whole device, cut to
// the serving engine's share of the SMs.
int serve_sparse_grid(const Serve* sv, int grid)
{
    if (sv->sms <= 0 || sv->sparse_sms >= sv->sms) return grid;
    const int g = (int)((int64_t)grid * sv->sparse_sms / sv->sms);
    return g > 0 ? g : 1;
}

void serve_delete(Serve* sv) { delete sv; }

// Set the ring up on first use; false when it is unavailable (then every
// request takes its own stream).
bool serve_ring_init(mars_ctx* c, Serve* sv)
{
    if (sv->ring) return true;
    if (!env_flag("MARS_SERVE_RING", 1) || !plan_serve_ring(c->device, &sv->plan)) return false;
    sv->plan.grid = serve_sparse_grid(sv, sv->plan.grid);
    bool ok = cudaMalloc((void**)&sv->ring, sizeof(ServeRing)) == cudaSuccess &&
              cudaMemset(sv->ring, 0, sizeof(ServeRing)) == cudaSuccess &&
              cudaMallocHost((void**)&sv->stage_jobs, sizeof(BatchJob) * kRingCap) == cudaSuccess &&
              cudaMallocHost((void**)&sv->stage_slots, sizeof(RingSlot) * kRingCap) == cudaSuccess &&
              cudaMallocHost((void**)&sv->stage_tail, sizeof(int32_t) * kRingCap) == cudaSuccess &&
              cudaHostAlloc((void**)&sv->done, sizeof(int32_t) * kRingCap, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void**)&sv->done_dev, sv->done, 0) == cudaSuccess &&
              cudaStreamCreateWithFlags(&sv->pub_st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&sv->ring_st, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&sv->ring_ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaDeviceSynchronize() == cudaSuccess;
    if (ok) std::memset(sv->done, 0, sizeof(int32_t) * kRingCap);
    sv->ring_on = ok;
    return ok;
}

void serve_ring_free(Serve* sv)
{
    if (sv->ring) {
        int32_t one = 1;
        cudaMemcpyAsync(&sv->ring->stop, &one, sizeof one, cudaMemcpyHostToDevice, sv->pub_st);
        cudaStreamSynchronize(sv->pub_st);
        cudaStreamSynchronize(sv->ring_st);
        cudaFree(sv->ring);
        sv->ring = nullptr;
    }
    if (sv->stage_jobs) cudaFreeHost(sv->stage_jobs);
    if (sv->stage_slots) cudaFreeHost(sv->stage_slots);
    if (sv->stage_tail) cudaFreeHost(sv->stage_tail);
    if (sv->done) cudaFreeHost(sv->done);
    if (sv->pub_st) cudaStreamDestroy(sv->pub_st);
    if (sv->ring_st) cudaStreamDestroy(sv->ring_st);
    if (sv->ring_ev) cudaEventDestroy(sv->ring_ev);
    sv->stage_jobs = nullptr;
    sv->stage_slots = nullptr;
    sv->stage_tail = nullptr;
    sv->done = nullptr;
    sv->pub_st = sv->ring_st = nullptr;
    sv->ring_ev = nullptr;
    sv->ring_on = false;
}

// Launch the serving kernel unless one is still running.
int serve_ring_ensure_kernel(mars_ctx* c, Serve* sv)
{
    if (sv->kernel_live) {
        const cudaError_t e = cudaEventQuery(sv->ring_ev);
        if (e == cudaErrorNotReady) return MARS_OK;
        if (e != cudaSuccess) return fail(c, MARS_EDEVICE, "serving kernel: %s", cudaGetErrorString(e));
        sv->kernel_live = false;
    }
    MARS_CUDA(c, launch_serve_ring(sv->ring, sv->plan, sv->idle_polls, sv->ring_st));
    MARS_CUDA(c, cudaEventRecord(sv->ring_ev, sv->ring_st));
    sv->kernel_live = true;
    return MARS_OK;
}

// Serving-ring jobs admitted at once, besides the in-flight limit of the
// other requests.
constexpr int kServeLight = 64;

bool serve_ring_init(mars_ctx* c, Serve* sv);

// Whether a request runs as a job of the persistent serving kernel: a
// sequential MARS solve of a sparse integer instance whose magnetisations fit
// on chip, while the ring has room.
bool serve_ring_eligible(mars_ctx* c, Serve* sv, const DevInstance& d, const mars_params& p)
{
    if (d.dense || !d.integer || p.update != MARS_UPDATE_GS || p.method != MARS_METHOD_MARS) return false;
    if (!serve_ring_init(c, sv) || sv->tail >= kRingCap) return false;
    int rt = 1;
    return ring_job_format(d, sv->plan, &rt) >= 0;
}

Serve* serve_get(mars_ctx* c)
{
    if (!c->serve) {
        c->serve = std::unique_ptr<Serve, void (*)(Serve*)>(new Serve(), serve_delete);
        Serve* nv = c->serve.get();
        cudaDeviceGetAttribute(&nv->sms, cudaDevAttrMultiProcessorCount, c->device);
        nv->sparse_sms = std::max(1, std::min(nv->sms, env_flag("MARS_SERVE_SPARSE_SMS", nv->sms / 2)));
    }
    Serve* sv = c->serve.get();
    while ((int)sv->streams.size() < sv->max_inflight) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) break;
        sv->free_slots.push_back((int)sv->streams.size());
        sv->streams.push_back(st);
    }
    return sv;
}

struct PinnedView {
    DevResult* res;
    int32_t* status;
    int32_t* counters;
    int8_t* best;
};

PinnedView pinned_view(unsigned char* base)
{
    PinnedView v;
    v.res = (DevResult*)base;
    v.status = (int32_t*)(base + 128);
    v.counters = (int32_t*)(base + 192);
    v.best = (int8_t*)(base + 256);
    return v;
}

void serve_free_req(mars_ctx* c, Serve* sv, ServeReq* q)
{
    if (q->ring_job >= 0) {
        sv->ring_refs -= 1;
        q->ring_job = -1;
    }
    if (q->st) {
        for (auto& b : q->bufs) dev_free_on(c, &b, q->st);
        q->bufs.clear();
    }
    if (q->pinned) {
        cudaFreeHost(q->pinned);
        q->pinned = nullptr;
    }
    if (q->ev) {
        cudaEventDestroy(q->ev);
        q->ev = nullptr;
    }
    if (q->slot >= 0) {
        sv->free_slots.push_back(q->slot);
        (q->light ? sv->light_inflight : sv->inflight) -= 1;
        q->slot = -1;
    }
    q->tc.reset();
}

// Device bytes a request holds while it runs (what admission checks): an
// upper bound on what serve_launch and tc_setup allocate for it, from the same
// plans they use, so that an admitted request never meets the budget check
// half-way through its set-up.
size_t serve_footprint(const DevInstance& d, const mars_params& p, int device)
{
    const size_t R = (size_t)p.replicas, n = (size_t)d.n;
    const bool jacobi = p.update == MARS_UPDATE_JACOBI || p.method == MARS_METHOD_NMFA;
    // t0, sigma, energies (double and int64), sweeps/levels/capped, the work
    // counter and status, the result record, the best spins, and the replica
    // queue at its widest slot rounding (at most 8 replicas per tile)
    size_t b = R * 4 + R * n + R * 16 + R * 12 + 8 + sizeof(DevResult) + n + (R + 8) * 4;
    if (d.dense && (p.precision == MARS_BF16 || p.precision == MARS_FP8)) {
        const size_t np = (size_t)d.n_pad, Rp = (R + 127) / 128 * 128;
        b += R * np * 4;                                            // S, FP32
        b += Rp * np * (p.precision == MARS_FP8 ? 1 : 2);           // its low-precision copy
        b += 2 * (size_t)kChainMaxSplit * Rp * 128 * 4;             // split-K partials, two buffers
        b += 2 * Rp * 128 * 4;                                      // next-panel fields
        b += R * (8 + 4 + 4 + 5 * 4) + 16;                          // per-slot state, counters
        b += (2 * (size_t)kTcMaxBatch * (np / 128) + 1) * 4;        // persistent batches' counters
    } else if (d.dense) {
        const DensePlan dp = plan_dense(d, (int)R, jacobi ? 1 : 0, device);
        b += dp.scratch_floats * sizeof(float);
    } else {
        // the serving ring needs no scratch; the stream route takes its plan's
        SparsePlan sp;
        if (jacobi || !plan_sparse_sell(d, (int)R, device, &sp)) sp = plan_sparse(d, (int)R, jacobi ? 1 : 0, device);
        b += sp.scratch_floats * sizeof(float);
    }
    return b;
}

// The request's results to pinned memory, then its event.
int serve_copy_results(mars_ctx* c, ServeReq* q)
{
    cudaStream_t st = q->st;
    PinnedView v = pinned_view(q->pinned);
    MARS_CUDA(c, cudaMemcpyAsync(v.res, q->dres, sizeof(DevResult), cudaMemcpyDeviceToHost, st));
    MARS_CUDA(c, cudaMemcpyAsync(v.status, q->s.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MARS_CUDA(c, cudaMemcpyAsync(v.best, q->dbest, q->dev.n, cudaMemcpyDeviceToHost, st));
    MARS_CUDA(c, cudaEventRecord(q->ev, st));
    q->state = ReqState::Finishing;
    return MARS_OK;
}

int serve_finish_enqueue(mars_ctx* c, ServeReq* q)
{
    cudaStream_t st = q->st;
    if (!q->dev.integer && q->dev.exact_ok)
        MARS_CUDA(c, launch_energy(q->dev, q->s.sigma, q->s.R, q->s.energy, nullptr, q->s.status, st));
    MARS_CUDA(c, launch_best(q->s, q->dev.n, q->dev.integer, q->dbest, q->dres, st));
    return serve_copy_results(c, q);
}

// Allocate, enqueue the whole pipeline (or the first batch of a tensor-core
// descent) on the request's stream, and record its event.
int serve_launch(mars_ctx* c, Serve* sv, ServeReq* q)
{
    Instance* in = find(c, q->inst);
    if (!in) return fail(c, MARS_ENOTFOUND, "instance %d was freed before its request ran", q->inst);
    q->dev = in->dev;
    q->total_weight = in->info.total_weight;
    q->err_bound = (in->dev.integer || in->dev.exact_ok)
                       ? 0.0
                       : std::ldexp(in->abs_weight, -53) * (double)(in->info.nnz / 2 + in->dev.n);
    if (sv->free_slots.empty()) {
        cudaStream_t ns;
        MARS_CUDA(c, cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking));
        sv->free_slots.push_back((int)sv->streams.size());
        sv->streams.push_back(ns);
    }
    q->slot = sv->free_slots.back();
    sv->free_slots.pop_back();
    (q->light ? sv->light_inflight : sv->inflight) += 1;
    q->st = sv->streams[q->slot];
    cudaStream_t st = q->st;
    const mars_params& p = q->p;
    const int32_t R = p.replicas, n = q->dev.n;
    int rc;
    size_t held = 0;
    auto get = [&](size_t bytes, void** out) -> int {
        held += bytes;
        if (held > q->footprint)
            return fail(c, MARS_EDEVICE, "internal: request %lld allocates more than its admission bound %zu",
                        (long long)q->id, q->footprint);
        DevMem m;
        int r = dev_alloc_on(c, bytes, &m, st);
        if (r) return r;
        q->bufs.push_back(m);
        *out = m.p;
        return MARS_OK;
    };
    MARS_CUDA(c, cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming));
    MARS_CUDA(c, cudaMallocHost((void**)&q->pinned, 256 + (size_t)n));
    DevSolve& s = q->s;
    s.R = R;
    s.seed = p.seed;
    s.stream = p.stream;
    s.c_step = p.c_step;
    s.d_min = (float)p.d_min;
    s.k_max = p.k_max;
    s.fixed_sweeps = p.fixed_sweeps;
    set_schedule(s, &p);
    s.jacobi = p.update == MARS_UPDATE_JACOBI;
    set_method(s, &p);
    s.m0 = p.m0;
    float* t0 = nullptr;
    if ((rc = get((size_t)R * sizeof(float), (void**)&t0))) return rc;
    if (p.t0) {
        MARS_CUDA(c, cudaMemcpyAsync(t0, p.t0, R * sizeof(float), cudaMemcpyDeviceToDevice, st));
    } else {
        MARS_CUDA(c, launch_draw(p.seed, p.stream, 0, R, 0, p.t_min, p.t_max, nullptr, t0, st));
    }
    s.t0 = t0;
    if ((rc = get((size_t)R * n, (void**)&s.sigma))) return rc;
    if ((rc = get((size_t)R * sizeof(double), (void**)&s.energy))) return rc;
    if ((rc = get((size_t)R * sizeof(long long), (void**)&s.energy_i64))) return rc;
    if ((rc = get((size_t)R * sizeof(int32_t), (void**)&s.sweeps))) return rc;
    if ((rc = get((size_t)R * sizeof(int32_t), (void**)&s.levels))) return rc;
    if ((rc = get((size_t)R * sizeof(int32_t), (void**)&s.capped))) return rc;
    if ((rc = get(2 * sizeof(int32_t), (void**)&s.work_counter))) return rc;
    s.status = s.work_counter + 1;
    if ((rc = get(sizeof(DevResult), (void**)&q->dres))) return rc;
    if ((rc = get((size_t)n, (void**)&q->dbest))) return rc;
    const bool tc = q->dev.dense && (p.precision == MARS_BF16 || p.precision == MARS_FP8);
    int rt = 1;
    SparsePlan sp;
    DensePlan dp;
    if (tc) {
        rt = 1;
    } else if (q->dev.dense) {
        dp = plan_dense(q->dev, R, s.jacobi, c->device);
        if (dp.scratch_floats && (rc = get(dp.scratch_floats * sizeof(float), (void**)&s.m_scratch))) return rc;
    } else {
        // the serving ring: one persistent kernel for every sparse request
        // (integer couplings: the kernel's fused int64 energies are final, so
        // the job needs no kernel after the serving kernel)
        int job_rt = 1;
        const int fmt = !s.jacobi && q->dev.integer && serve_ring_init(c, sv)
                            ? ring_job_format(q->dev, sv->plan, &job_rt)
                            : -1;
        const int k = (int)sv->tail;
        if (fmt >= 0 && sv->tail < kRingCap) {
            const int32_t rr = job_rt;
            const int32_t ntiles = (R + rr - 1) / rr;
            int32_t* queue = nullptr;
            if ((rc = get((size_t)ntiles * rr * sizeof(int32_t), (void**)&queue))) return rc;
            MARS_CUDA(c, launch_queue_identity(queue, ntiles * rr, R, s.work_counter, st));
            s.tile_rep = queue;
            s.ntiles = ntiles;
            s.rt = rr;
            // the job's counters and flag live in the ring
            s.work_counter = &sv->ring->slots[k].taken;
            s.status = &sv->ring->slots[k].status;
            s.finished = &sv->ring->slots[k].finished;
            s.done_flag = sv->done_dev + k;
            s.res = q->dres;
            s.best_out = q->dbest;
            sv->done[k] = 0;
            BatchJob job;
            job.in = q->dev;
            job.s = s;
            job.fmt = fmt;
            job.rt = job_rt;
            sv->stage_jobs[k] = job;
            sv->stage_slots[k] = RingSlot{};
            sv->stage_tail[k] = (int32_t)(sv->tail + 1);
            // publish after the request's own set-up (start temperatures, queue)
            MARS_CUDA(c, cudaEventRecord(q->ev, st));
            MARS_CUDA(c, cudaStreamWaitEvent(sv->pub_st, q->ev, 0));
            MARS_CUDA(c, cudaMemcpyAsync(&sv->ring->jobs[k], &sv->stage_jobs[k], sizeof(BatchJob),
                                         cudaMemcpyHostToDevice, sv->pub_st));
            MARS_CUDA(c, cudaMemcpyAsync(&sv->ring->slots[k], &sv->stage_slots[k], sizeof(RingSlot),
                                         cudaMemcpyHostToDevice, sv->pub_st));
            MARS_CUDA(c, cudaMemcpyAsync(&sv->ring->tail, &sv->stage_tail[k], sizeof(int32_t),
                                         cudaMemcpyHostToDevice, sv->pub_st));
            q->ring_job = sv->tail;
            sv->ring_refs += 1;
            sv->tail += 1;
            sv->ring_jobs += 1;
            q->state = ReqState::RingRunning;
            return serve_ring_ensure_kernel(c, sv);
        }
        if (s.jacobi || !plan_sparse_sell(q->dev, R, c->device, &sp))
            sp = plan_sparse(q->dev, R, s.jacobi, c->device);
        sp.grid = serve_sparse_grid(sv, sp.grid);  // the per-CTA buffers below follow the grid
        rt = sp.rt;
        float* scr = nullptr;
        if (sp.scratch_floats && (rc = get(sp.scratch_floats * sizeof(float), (void**)&scr))) return rc;
        const size_t per = (size_t)sp.grid * n * rt;
        if (!sp.onchip) { s.m_scratch = scr; scr += per; }
        if (s.jacobi) s.m_next = scr;
    }
    const int32_t ntiles = (R + rt - 1) / rt;
    int32_t* queue = nullptr;
    if ((rc = get((size_t)ntiles * rt * sizeof(int32_t), (void**)&queue))) return rc;
    MARS_CUDA(c, launch_queue_identity(queue, ntiles * rt, R, s.work_counter, st));
    s.tile_rep = queue;
    s.ntiles = ntiles;
    s.rt = rt;
    if (tc) {
        q->tc.reset(new TcRun());
        TcRun* run = q->tc.get();
        const float t0_max = (float)std::max(p.t_max, 0.0);
        if ((rc = tc_setup(c, q->dev, s, queue, p.t0 ? 1e6f * (float)p.c_step : t0_max,
                           p.precision == MARS_FP8, st, get, run)))
            return rc;
        run->h_counters = pinned_view(q->pinned).counters;
        sv->stream_jobs += 1;
        if ((rc = tc_enqueue_batch(c, run, st))) return rc;
        MARS_CUDA(c, cudaEventRecord(q->ev, st));
        q->state = ReqState::TcRunning;
        return MARS_OK;
    }
    sv->stream_jobs += 1;
    if (q->dev.dense) {
        MARS_CUDA(c, launch_dense(q->dev, s, dp, st));
    } else if (sp.sell) {
        MARS_CUDA(c, launch_sparse_sell(q->dev, s, sp, st));
    } else {
        MARS_CUDA(c, launch_sparse(q->dev, s, sp, st));
    }
    return serve_finish_enqueue(c, q);
}

void serve_mark_failed(mars_ctx* c, Serve* sv, ServeReq* q, int rc)
{
    q->rc = rc;
    q->err = c->err;
    q->state = ReqState::Failed;
    serve_free_req(c, sv, q);
}

void serve_progress(mars_ctx* c)
{
    Serve* sv = serve_get(c);
    // collect
    bool ring_pending = false;
    for (auto& kv : sv->reqs) {
        ServeReq* q = kv.second.get();
        if (q->state == ReqState::RingRunning) {
            const int k = (int)q->ring_job;
            if (*reinterpret_cast<volatile int32_t*>(sv->done + k)) {
                const int rc = serve_copy_results(c, q);  // the kernel already selected the best
                if (rc) serve_mark_failed(c, sv, q, rc);
            } else {
                ring_pending = true;
            }
            continue;
        }
        if (q->state != ReqState::TcRunning && q->state != ReqState::Finishing) continue;
        const cudaError_t e = cudaEventQuery(q->ev);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) {
            fail(c, MARS_EDEVICE, "CUDA error: %s", cudaGetErrorString(e));
            serve_mark_failed(c, sv, q, MARS_EDEVICE);
            continue;
        }
        if (q->state == ReqState::TcRunning && q->cancelled) {
            // its last batch has ended: no more sweeps
            fail(c, MARS_ECANCELED, "request %lld was cancelled", (long long)q->id);
            serve_mark_failed(c, sv, q, MARS_ECANCELED);
            continue;
        }
        if (q->state == ReqState::TcRunning) {
            const int r = tc_after_batch(c, q->tc.get());
            int rc = MARS_OK;
            if (r < 0) {
                rc = r;
            } else if (r == 1) {
                rc = tc_enqueue_batch(c, q->tc.get(), q->st);
                if (!rc && cudaEventRecord(q->ev, q->st) != cudaSuccess) rc = MARS_EDEVICE;
            } else {
                rc = launch_tc_finalize(q->tc->t, q->dev, q->s, q->st) == cudaSuccess ? MARS_OK : MARS_EDEVICE;
                if (!rc) rc = serve_finish_enqueue(c, q);
            }
            if (rc) serve_mark_failed(c, sv, q, rc);
            continue;
        }
        // Finishing: results are in pinned memory
        PinnedView v = pinned_view(q->pinned);
        if (*v.status != kDevOk) {
            fail(c, MARS_EDEVICE, "device status %d", *v.status);
            serve_mark_failed(c, sv, q, MARS_EDEVICE);
            continue;
        }
        q->state = ReqState::Done;
        if (q->ring_job >= 0) {
            sv->ring_refs -= 1;
            q->ring_job = -1;
        }
        if (q->cancelled) {
            fail(c, MARS_ECANCELED, "request %lld was cancelled", (long long)q->id);
            serve_mark_failed(c, sv, q, MARS_ECANCELED);
            continue;
        }
        for (auto& b : q->bufs) dev_free_on(c, &b, q->st);
        q->bufs.clear();
        if (q->slot >= 0) {
            sv->free_slots.push_back(q->slot);
            (q->light ? sv->light_inflight : sv->inflight) -= 1;
            q->slot = -1;
        }
    }
    // a published job is always taken up: relaunch the serving kernel if it
    // went idle and exited before the job's tail reached it
    if (ring_pending) {
        const int rc = serve_ring_ensure_kernel(c, sv);
        if (rc) {
            for (auto& kv : sv->reqs)
                if (kv.second->state == ReqState::RingRunning) serve_mark_failed(c, sv, kv.second.get(), rc);
        }
    }
    // reset the ring once its kernel has exited and no request reads a slot
    if (sv->ring && sv->tail > 0 && sv->ring_refs == 0) {
        const bool live = sv->kernel_live && cudaEventQuery(sv->ring_ev) == cudaErrorNotReady;
        if (!live) {
            sv->kernel_live = false;
            if (cudaMemsetAsync(sv->ring, 0, sizeof(ServeRing), sv->pub_st) == cudaSuccess) {
                std::memset(sv->done, 0, sizeof(int32_t) * kRingCap);
                sv->tail = 0;
            }
        }
    }
    // admit: serving-ring jobs (small sparse requests) whenever fewer than
    // kServeLight are in flight, passing requests queued before them; the
    // others in arrival order while fewer than max_inflight of them run. Both
    // wait for the HBM budget.
    bool heavy_blocked = false;
    for (auto qi = sv->queue.begin(); qi != sv->queue.end();) {
        auto it = sv->reqs.find(*qi);
        if (it == sv->reqs.end()) { qi = sv->queue.erase(qi); continue; }
        ServeReq* q = it->second.get();
        Instance* in = find(c, q->inst);
        if (!in) {
            qi = sv->queue.erase(qi);
            fail(c, MARS_ENOTFOUND, "instance %d was freed before its request ran", q->inst);
            serve_mark_failed(c, sv, q, MARS_ENOTFOUND);
            continue;
        }
        const bool light = serve_ring_eligible(c, sv, in->dev, q->p);
        if (light ? sv->light_inflight >= kServeLight : heavy_blocked || sv->inflight >= sv->max_inflight) {
            heavy_blocked |= !light;
            ++qi;
            continue;
        }
        const size_t need = serve_footprint(in->dev, q->p, c->device);
        if (c->budget && c->used + need > c->budget) {
            if (sv->inflight + sv->light_inflight == 0) {  // it will never fit
                qi = sv->queue.erase(qi);
                fail(c, MARS_ENOMEM, "request needs about %zu bytes; the HBM budget is %zu", need, c->budget);
                serve_mark_failed(c, sv, q, MARS_ENOMEM);
                continue;
            }
            heavy_blocked |= !light;  // wait for memory to free up
            ++qi;
            continue;
        }
        qi = sv->queue.erase(qi);
        q->footprint = need;
        q->light = light;
        const int rc = serve_launch(c, sv, q);
        if (rc) serve_mark_failed(c, sv, q, rc);
    }
}

void serve_release(mars_ctx* c)
{
    if (!c->serve) return;
    Serve* sv = c->serve.get();
    serve_ring_free(sv);
    for (cudaStream_t st : sv->streams) cudaStreamSynchronize(st);
    for (auto& kv : sv->reqs) serve_free_req(c, sv, kv.second.get());
    sv->reqs.clear();
    for (cudaStream_t st : sv->streams) cudaStreamDestroy(st);
    sv->streams.clear();
    c->serve.reset();
}


extern "C" {

int mars_serve_limits(mars_ctx* c, int32_t max_inflight)
{
    if (!c || max_inflight < 1 || max_inflight > 64) return MARS_EINVAL;
    DeviceGuard g(c->device);
    Serve* sv = serve_get(c);
    sv->max_inflight = std::max(max_inflight, (int32_t)sv->inflight);
    serve_get(c);
    return MARS_OK;
}

int mars_submit(mars_ctx* c, int32_t id, const mars_params* p, int64_t* req)
{
    if (!c || !p || !req) return MARS_EINVAL;
    Instance* in = find(c, id);
    if (!in) return fail(c, MARS_ENOTFOUND, "unknown instance %d", id);
    if (p->replicas < 1 || !std::isfinite(p->t_min) || !std::isfinite(p->t_max) || p->t_min > p->t_max ||
        !(p->c_step > 0.0) || !schedule_ok(p) || levels_bound(p, p->t_max) > kMaxLevels ||
        !(p->d_min >= 0.0) ||
        p->k_max < 1 || p->fixed_sweeps < 0 ||
        (p->update != MARS_UPDATE_GS && p->update != MARS_UPDATE_JACOBI))
        return fail(c, MARS_EINVAL, "bad parameters");
    if (const char* e = method_error(p)) return fail(c, MARS_EINVAL, "%s", e);
    const bool tc = p->precision == MARS_BF16 || p->precision == MARS_FP8;
    if (p->precision != MARS_FP32 && !(tc && in->dev.dense && p->update == MARS_UPDATE_GS))
        return fail(c, MARS_EINVAL, "precision %d is not available for this instance", p->precision);
    if (p->precision == MARS_FP8 && !in->dev.J8)
        return fail(c, MARS_EINVAL, "FP8 needs integer couplings exactly representable in E4M3");
    if ((p->m0 || p->t0) && !(p->flags & MARS_DEVICE_PTR))
        return fail(c, MARS_EINVAL, "served requests take m0/t0 as device pointers");
    if (tc && p->t0) return fail(c, MARS_EINVAL, "served tensor-core requests draw t0 themselves");
    DeviceGuard g(c->device);
    Serve* sv = serve_get(c);
    auto q = std::make_unique<ServeReq>();
    q->id = sv->next_id++;
    q->inst = id;
    q->p = *p;
    *req = q->id;
    sv->queue.push_back(q->id);
    sv->reqs[q->id] = std::move(q);
    serve_progress(c);
    return MARS_OK;
}

int mars_poll(mars_ctx* c, int64_t req, int8_t* best_spins, mars_result* result)
{
    if (!c) return MARS_EINVAL;
    DeviceGuard g(c->device);
    serve_progress(c);
    Serve* sv = c->serve.get();
    auto it = sv ? sv->reqs.find(req) : std::map<int64_t, std::unique_ptr<ServeReq>>::iterator();
    if (!sv || it == sv->reqs.end()) return fail(c, MARS_ENOTFOUND, "unknown request %lld", (long long)req);
    ServeReq* q = it->second.get();
    if (q->state == ReqState::Failed) {
        const int rc = q->rc;
        c->err = q->err;
        sv->reqs.erase(it);
        return rc;
    }
    if (q->state != ReqState::Done) return MARS_EAGAIN;
    PinnedView v = pinned_view(q->pinned);
    if (best_spins) std::memcpy(best_spins, v.best, q->dev.n);
    if (result) {
        const DevResult& h = *v.res;
        std::memset(result, 0, sizeof *result);
        result->best_energy = h.best_energy;
        result->best_energy_i64 = h.best_energy_i64;
        result->best_cut = (q->total_weight - h.best_energy) / 2.0;
        result->best_replica = h.best_replica;
        result->hits = h.hits;
        result->mean_energy = h.sum_energy / q->p.replicas;
        result->sweeps = h.sweeps;
        result->spin_updates = h.sweeps * (int64_t)q->dev.n;
        result->levels = h.levels;
        result->capped_levels = h.capped;
        result->integer = q->dev.integer;
        result->energy_err_bound = q->err_bound;
        result->status = MARS_OK;
    }
    serve_free_req(c, sv, q);
    sv->reqs.erase(it);
    return MARS_OK;
}

int mars_cancel(mars_ctx* c, int64_t req)
{
    if (!c) return MARS_EINVAL;
    DeviceGuard g(c->device);
    Serve* sv = c->serve.get();
    auto it = sv ? sv->reqs.find(req) : std::map<int64_t, std::unique_ptr<ServeReq>>::iterator();
    if (!sv || it == sv->reqs.end()) return fail(c, MARS_ENOTFOUND, "unknown request %lld", (long long)req);
    ServeReq* q = it->second.get();
    switch (q->state) {
    case ReqState::Queued: {
        auto qi = std::find(sv->queue.begin(), sv->queue.end(), req);
        if (qi != sv->queue.end()) sv->queue.erase(qi);
        q->rc = MARS_ECANCELED;
        q->err = "request was cancelled before it ran";
        q->state = ReqState::Failed;
        break;
    }
    case ReqState::Done:  // finished but not collected: discard the results
        q->rc = MARS_ECANCELED;
        q->err = "request was cancelled";
        q->state = ReqState::Failed;
        serve_free_req(c, sv, q);
        break;
    case ReqState::Failed:
        break;
    default:  // on the GPU: its kernels finish, then it is dropped
        q->cancelled = true;
        break;
    }
    serve_progress(c);
    return MARS_OK;
}

int mars_serve_status(mars_ctx* c, int32_t* queued, int32_t* running)
{
    if (!c) return MARS_EINVAL;
    DeviceGuard g(c->device);
    serve_progress(c);
    Serve* sv = c->serve.get();
    if (queued) *queued = sv ? (int32_t)sv->queue.size() : 0;
    if (running) *running = sv ? sv->inflight + sv->light_inflight : 0;
    return MARS_OK;
}

int mars_serve_counters(mars_ctx* c, int64_t* ring_jobs, int64_t* stream_jobs)
{
    if (!c) return MARS_EINVAL;
    const Serve* sv = c->serve.get();
    if (ring_jobs) *ring_jobs = sv ? sv->ring_jobs : 0;
    if (stream_jobs) *stream_jobs = sv ? sv->stream_jobs : 0;
    return MARS_OK;
}

}  // extern "C"
