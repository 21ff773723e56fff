// Host side of the level-synchronous sparse descent (kernels_sparse_wide.cu):
// every replica resident in global memory, a sweep = one launch per level of
// the schedule and one decision launch (Section 3, Algorithm 1: the levels
// in order, then the stopping rule and the cooling step). Sweeps run in
// batches that double up to kTcMaxBatch sweeps: the first sweep of a batch is
// launched directly with its level launches timed, the rest replay one sweep
// captured as a CUDA graph; between batches the host reads the live replica
// count and stops at zero.
#include "mars_host.h"

#include <algorithm>
#include <cmath>

int run_sparse_wide(mars_ctx* c, const DevInstance& d, const mars_params* p, const DevSolve& s,
                    const WidePlan& wp, float t0_max, Scratch& S, int64_t* launches, LevelProfile* prof)
{
    cudaStream_t st = c->stream;
    int rc;
    DevWide w;
    w.rt = wp.rt;
    w.groups = wp.groups;
    w.slab = wp.slab;
    const size_t slots = (size_t)wp.groups * wp.rt;
    if ((rc = S.get((size_t)wp.groups * wp.slab, &w.m))) return rc;
    if ((rc = S.get(slots, &w.T))) return rc;
    if ((rc = S.get(slots, &w.invT))) return rc;
    if ((rc = S.get(slots, &w.live))) return rc;
    if ((rc = S.get(slots, &w.lvl_sweeps))) return rc;
    if ((rc = S.get(slots, &w.sweeps))) return rc;
    if ((rc = S.get(slots, &w.levels))) return rc;
    if ((rc = S.get(slots, &w.capped))) return rc;
    if ((rc = S.get(slots, &w.dmax))) return rc;
    if ((rc = S.get((size_t)wp.groups, &w.glist))) return rc;
    if ((rc = S.get(2, &w.counters))) return rc;
    MARS_CUDA(c, launch_wide_init(d, s, w, wp, st));
    MARS_CUDA(c, launch_wide_decide(s, w, 0, st));
    *launches += 2;

    // Most sweeps any replica can take: every level capped (a quench level
    // keeps the stopping rule even when the others run fixed sweeps).
    const double lv = levels_bound(p, t0_max) + 2.0;
    const int64_t cap = (int64_t)(lv * (double)std::max(s.fixed_sweeps, s.k_max)) + 1;

    int32_t* h = nullptr;
    MARS_CUDA(c, cudaMallocHost((void**)&h, 2 * sizeof(int32_t)));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cudaFreeHost(h);
    };
    auto check = [&](cudaError_t e, const char* what) -> int {
        if (e == cudaSuccess) return MARS_OK;
        cleanup();
        return fail(c, MARS_EDEVICE, "%s failed: %s", what, cudaGetErrorString(e));
    };
    if ((rc = check(cudaMemcpyAsync(h, w.counters, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
                    "counter copy")))
        return rc;
    if ((rc = check(cudaStreamSynchronize(st), "descent start"))) return rc;

    // one sweep: the levels in order, then the decision
    if ((rc = check(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "sweep capture"))) return rc;
    cudaError_t le = cudaSuccess;
    for (int l = 0; l < d.nlev && le == cudaSuccess; ++l) le = launch_wide_level(d, s, w, wp, l, st);
    if (le == cudaSuccess) le = launch_wide_decide(s, w, 1, st);
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if ((rc = check(le, "level launch"))) return rc;
    if ((rc = check(ce, "sweep capture"))) return rc;
    if ((rc = check(cudaGraphInstantiate(&exec, graph, 0), "sweep graph"))) return rc;

    while ((int)c->prof.size() < 2 * d.nlev) {
        cudaEvent_t e;
        if ((rc = check(cudaEventCreate(&e), "event"))) return rc;
        c->prof.push_back(e);
    }
    int64_t done = 0;
    int batch = 1;
    while (h[1] > 0) {
        if (done > cap) {
            cleanup();
            return fail(c, MARS_EDEVICE, "descent exceeded its sweep bound");
        }
        const int64_t live = h[1];
        // the batch's first sweep, each level launch timed
        for (int l = 0; l < d.nlev; ++l) {
            if ((rc = check(cudaEventRecord(c->prof[2 * l], st), "event"))) return rc;
            if ((rc = check(launch_wide_level(d, s, w, wp, l, st), "level launch"))) return rc;
            if ((rc = check(cudaEventRecord(c->prof[2 * l + 1], st), "event"))) return rc;
        }
        if ((rc = check(launch_wide_decide(s, w, 1, st), "decision launch"))) return rc;
        for (int b = 1; b < batch; ++b)
            if ((rc = check(cudaGraphLaunch(exec, st), "sweep graph launch"))) return rc;
        if ((rc = check(cudaMemcpyAsync(h, w.counters, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
                        "counter copy")))
            return rc;
        if ((rc = check(cudaStreamSynchronize(st), "sweeps"))) return rc;
        for (int l = 0; l < d.nlev; ++l) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, c->prof[2 * l], c->prof[2 * l + 1]);
            prof->seconds += ms * 1e-3;
        }
        prof->launches += d.nlev;
        prof->updates += live * (int64_t)d.n;
        done += batch;
        *launches += (int64_t)batch * (d.nlev + 1);
        batch = std::min(batch * 2, kTcMaxBatch);
    }
    cleanup();
    MARS_CUDA(c, launch_wide_finalize(d, s, w, wp, st));
    *launches += 1;
    return MARS_OK;
}
