// The dense descent on tensor cores, host side: device state and tensor
// maps of a descent, one sweep as a sequence of panel GEMMs and in-panel
// chains (captured once as a CUDA graph and replayed), batches of sweeps with
// the active count read back between them, and the blocking descent of
// mars_solve. The kernels are in kernels_dense_tc.cu.
#include "mars_host.h"

#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

using namespace mars;

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
        cudaGetLastError();
    }
    return fn;
}

// Row-major [outer][inner] BF16 matrix, boxes of box_inner x box_outer with the
// 128-byte swizzle (box_inner = 64 BF16 = 128 bytes).
// 2-D K-major operand map: inner (K) extent `inner` elements of `elem` bytes,
// `outer` rows, 128-byte swizzled boxes of box_inner x box_outer.
bool encode_2d(CUtensorMap* m, CUtensorMapDataType dt, uint32_t elem, const void* base, uint64_t inner,
               uint64_t outer, uint32_t box_inner, uint32_t box_outer)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {inner * elem};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}



// The sweep's launch plan for `active` active replicas whose slots lie below
// `prefix`: replicas per chain warp, the GEMM schedule (plain, overlapped with
// the previous panel's chain, or panel pairs) and the split of K.
//
// With (nearly) every replica active the GEMMs fill the GPU and panel pairs
// win: they stream the magnetisations' copy once per two panels. Once fewer
// replicas remain the SMs are no longer all busy, so panel p+1's GEMM runs
// beside panel p's chain (the overlap) and the chain's steps are shortened by
// fewer replicas per warp; most of a solve's sweeps run in that regime (the
// replicas' sweep counts spread evenly from zero to the longest). K is split
// until one GEMM wave covers the SMs. A knob the instance's shape or an
// environment override fixes is kept. A plan change drops the captured
// sweep graph; the next batch captures the new one.
int tc_plan(mars_ctx* c, TcRun* run, int32_t active, int32_t prefix)
{
    // the count the defaults follow: the active replicas, or (a knob fixed)
    // the replica count, as measured for whole sweeps at N = 8192
    const int A = run->adaptive && active > 0 ? active : run->t.R;
    int rpw, ov, pair;
    if (run->adaptive) {
        // fastest all-active sweeps measured on a GB300 at N = 8192 (ms):
        // A = 4096 pairs/4 2.15; 2048 pairs/2 1.48; 1024 overlap/2 1.19;
        // 512 and below overlap/1 1.04-1.06
        rpw = A >= 3072 ? 4 : A >= 768 ? 2 : 1;
        ov = A < 1536 ? 1 : 0;
        pair = A >= 1536 ? 1 : 0;
    } else {
        rpw = A >= 2048 ? 4 : A >= 512 ? 2 : 1;
        ov = A >= 512 && A < 2048 ? 1 : 0;
        pair = A >= 2048 ? 1 : 0;
    }
    if (run->fixed_rpw >= 0) rpw = run->fixed_rpw;
    if (run->fixed_overlap >= 0) ov = run->fixed_overlap;
    if (run->fixed_pair >= 0) pair = run->fixed_pair;
    if (rpw != 1 && rpw != 2 && rpw != 4) rpw = 1;
    const bool pr = run->P >= 2 && pair != 0;
    const bool ovl = run->P >= 2 && ov != 0 && !pr;
    const int slots = std::min(std::max(prefix, 1), run->t.R);
    const int tiles = (slots + kTcBN - 1) / kTcBN;
    int splitk = 1;
    const int split_max = env_flag("MARS_TC_SPLITK_MAX", 16);
    const int wave = env_flag("MARS_TC_WAVE_PCT", 100) * run->sms / 100;  // CTAs one GEMM may use
    while (splitk < split_max && splitk * 2 <= kChainMaxSplit / rpw && tiles * splitk * 2 <= wave &&
           run->kblocks_total % (splitk * 2) == 0)
        splitk *= 2;
    const int chain_slots = std::min(tiles * kTcBN, run->t.R);  // the chains cover [0, chain_slots)
    // Persistent batches once the active replicas leave SMs free: chain CTAs
    // for every replica group (one group each) beside GEMM CTAs for the
    // panel's (tile, split) items, all resident (measured on a GB300 at
    // N = 8192 against the launched sweeps above).
    if (run->adaptive && run->allow_persist && run->P >= 2 && A <= env_flag("MARS_TC_PERSIST_MAX", 2048) &&
        run->flags) {
        const int prpw = A <= 512 ? 1 : A <= 1024 ? 2 : 4;
        TcPersist q;
        q.chain_items = (chain_slots + 8 * prpw - 1) / (8 * prpw);
        q.n_chain = std::min(q.chain_items, run->sms - 16);
        q.gemm_tiles = tiles;
        q.splitk = 1;
        while (q.splitk * 2 <= kChainMaxSplit / prpw && tiles * q.splitk * 2 <= run->sms - q.n_chain &&
               run->kblocks_total % (q.splitk * 2) == 0)
            q.splitk *= 2;
        q.n_gemm = std::min(tiles * q.splitk, run->sms - q.n_chain);
        q.P = run->P;
        // every replica group and every GEMM item has a CTA of its own
        if (q.n_chain >= 1 && q.n_gemm >= 1 && q.chain_items <= q.n_chain && tiles * q.splitk <= q.n_gemm) {
            if (run->exec) cudaGraphExecDestroy(run->exec);
            if (run->graph) cudaGraphDestroy(run->graph);
            run->exec = nullptr;
            run->graph = nullptr;
            run->persist = true;
            run->rpw = prpw;
            run->overlap = true;
            run->pair = false;
            run->splitk = q.splitk;
            run->t.splitk = q.splitk;
            run->g.kblocks = run->kblocks_total / q.splitk;
            run->gemm_tiles = tiles;
            run->chain_slots = chain_slots;
            q.G[0] = run->Gbuf[0];
            q.G[1] = run->Gbuf[1];
            q.Gx[0] = run->Gx[0];
            q.Gx[1] = run->Gx[1];
            q.gemm_done = run->flags;
            q.chain_done = run->flags + kTcMaxBatch * run->P;
            q.abort = run->flags + 2 * kTcMaxBatch * run->P;
            int khz = 0;
            cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c->device);
            q.spin_budget = 10LL * (khz > 0 ? khz : 2000000) * 1000;  // about ten seconds
            run->pp = q;
            return MARS_OK;
        }
    }
    run->persist = false;
    // Four warps per chain CTA when those CTAs fit in half of the SMs: with
    // two warps per scheduler the 128-step chain is partly issue-bound (on a
    // GB300 at N = 8192 with 128 replicas active a step took 55 ns with 8
    // warps per CTA and 42 ns with 4); with more replicas the extra CTAs
    // crowd out the GEMM (1024 active: 12.8 against 18.1 us per panel).
    int cw = (chain_slots + 4 * rpw - 1) / (4 * rpw) <= run->sms / 2 ? 4 : 8;
    if (const int f = env_flag("MARS_TC_CHAIN_WARPS", 0); f == 4 || f == 8) cw = f;
    if (run->exec && rpw == run->rpw && ovl == run->overlap && pr == run->pair && splitk == run->splitk &&
        tiles == run->gemm_tiles && chain_slots == run->chain_slots && cw == run->chain_warps)
        return MARS_OK;
    if (run->exec) cudaGraphExecDestroy(run->exec);
    if (run->graph) cudaGraphDestroy(run->graph);
    run->exec = nullptr;
    run->graph = nullptr;
    run->rpw = rpw;
    run->chain_warps = cw;
    run->overlap = ovl;
    run->pair = pr;
    run->splitk = splitk;
    run->t.splitk = splitk;
    run->g.kblocks = run->kblocks_total / splitk;
    run->gemm_tiles = tiles;
    run->chain_slots = chain_slots;
    if (ovl && !run->side) {
        MARS_CUDA(c, cudaStreamCreateWithFlags(&run->side, cudaStreamNonBlocking));
        run->ev.resize(1 + 2 * (size_t)run->P, nullptr);
        for (cudaEvent_t& e : run->ev) MARS_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    return MARS_OK;
}

// Device state of a tensor-core descent; buffers come from `get` so that the
// blocking path (Scratch) and the serving engine (per-request lists) can own them.
int tc_setup(mars_ctx* c, const DevInstance& d, const DevSolve& s, const int32_t* rep_dev,
             float t0_max, bool fp8, cudaStream_t st, const TcGet& get, TcRun* run)
{
    int rc;
    TcState& t = run->t;
    const int32_t R = s.R, n = d.n, n_pad = d.n_pad;
    const int32_t R_pad = (R + kTcBN - 1) / kTcBN * kTcBN;
    run->P = n_pad / 128;
    run->ntiles = R_pad / kTcBN;
    // The launch plan (replicas per chain warp, GEMM schedule, split of K)
    // follows the active replicas batch by batch (tc_plan) unless the
    // instance's shape (mars_set_shape, mars_autotune) or an environment
    // override fixes a knob.
    const LaunchShape& sh = d.shape;
    run->fixed_rpw = sh.tc_rpw >= 0 ? sh.tc_rpw : env_flag("MARS_TC_RPW", -1);
    run->fixed_overlap = sh.tc_overlap >= 0 ? sh.tc_overlap : env_flag("MARS_TC_OVERLAP", -1);
    run->fixed_pair = sh.tc_pair >= 0 ? sh.tc_pair : env_flag("MARS_TC_PAIR", -1);
    run->adaptive = run->fixed_rpw < 0 && run->fixed_overlap < 0 && run->fixed_pair < 0;
    run->sms = c->sms;
    run->kblocks_total = n_pad / (fp8 ? 128 : 64);
    t.R = R;
    t.R_pad = R_pad;
    t.n = n;
    t.n_pad = n_pad;
    t.Jdiag = d.Jdiag;
    t.Jsup = d.Jsup;
    t.h = d.h;
    t.new2old = d.new2old;
    t.m0 = s.m0;
    t.t0 = s.t0;
    t.seed = s.seed;
    t.stream = s.stream;
    t.c_step = s.c_step;
    t.d_min = s.d_min;
    t.k_max = s.k_max;
    t.fixed_sweeps = s.fixed_sweeps;
    t.geometric = s.geometric;
    t.quench = s.quench;
    t.cool_ratio = s.cool_ratio;
    t.t_floor = s.t_floor;
    t.rep = rep_dev;
    if ((rc = get((size_t)R * n_pad * sizeof(float), (void**)&t.S))) return rc;
    if (fp8 && !d.J8) return fail(c, MARS_EINVAL, "FP8 needs couplings exact in E4M3");
    if (fp8) {
        if ((rc = get((size_t)R_pad * n_pad, (void**)&t.S8))) return rc;
    } else if ((rc = get((size_t)R_pad * n_pad * sizeof(__nv_bfloat16), (void**)&t.Sb))) {
        return rc;
    }
    // split-K partials at the largest split any plan may take, two buffers
    run->g_floats_max = (size_t)kChainMaxSplit * R_pad * 128;
    if ((rc = get(2 * run->g_floats_max * sizeof(float), (void**)&t.G))) return rc;
    run->Gbuf[0] = t.G;
    run->Gbuf[1] = t.G + run->g_floats_max;
    {
        float* gx = nullptr;
        if ((rc = get(2 * (size_t)R_pad * 128 * sizeof(float), (void**)&gx))) return rc;
        run->Gx[0] = gx;
        run->Gx[1] = gx + (size_t)R_pad * 128;
    }
    // the persistent batches' counters, when cooperative launches are available
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
    if (coop && (rc = get((2 * (size_t)kTcMaxBatch * run->P + 1) * sizeof(int32_t), (void**)&run->flags)))
        return rc;
    if ((rc = get((size_t)R * sizeof(double), (void**)&t.T))) return rc;
    if ((rc = get((size_t)R * sizeof(float), (void**)&t.invT))) return rc;
    if ((rc = get((size_t)R * sizeof(float), (void**)&t.d))) return rc;
    if ((rc = get((size_t)R * sizeof(int32_t), (void**)&t.active))) return rc;
    if ((rc = get((size_t)R * sizeof(int32_t), (void**)&t.levels))) return rc;
    if ((rc = get((size_t)R * sizeof(int32_t), (void**)&t.lvl_sweeps))) return rc;
    if ((rc = get((size_t)R * sizeof(int32_t), (void**)&t.sweeps))) return rc;
    if ((rc = get((size_t)R * sizeof(int32_t), (void**)&t.capped))) return rc;
    if ((rc = get(4 * sizeof(int32_t), (void**)&t.counters))) return rc;
    if (fp8)
        MARS_CUDA(c, cudaMemsetAsync(t.S8, 0, (size_t)R_pad * n_pad, st));
    else
        MARS_CUDA(c, cudaMemsetAsync(t.Sb, 0, (size_t)R_pad * n_pad * sizeof(__nv_bfloat16), st));
    MARS_CUDA(c, cudaMemsetAsync(t.counters, 0, 4 * sizeof(int32_t), st));
    const bool maps_ok =
        fp8 ? encode_2d(&run->tmJ, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, d.J8, n_pad, n_pad, 128, 128) &&
                  encode_2d(&run->tmS, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, t.S8, n_pad, R_pad, 128, kTcBN)
            : encode_2d(&run->tmJ, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, d.Jbf, n_pad, n_pad, 64, 128) &&
                  encode_2d(&run->tmS, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, t.Sb, n_pad, R_pad, 64, kTcBN);
    if (!maps_ok) return fail(c, MARS_EDEVICE, "tensor map encoding failed");
    MARS_CUDA(c, launch_tc_init(t, st));
    MARS_CUDA(c, launch_tc_prefix(t, st));
    run->g.fp8 = fp8 ? 1 : 0;
    run->g.R_pad = R_pad;
    run->g.G = t.G;
    run->g.active_prefix = t.counters;
    run->g.err = t.counters + 2;
    // Every replica ends within (levels + 1) x (sweeps per level) sweeps.
    double levels_max = std::ceil((double)t0_max / s.c_step) + 1.0;
    if (s.geometric)
        levels_max = t0_max > s.t_floor ? std::ceil(std::log(s.t_floor / t0_max) / std::log(s.cool_ratio)) + 1.0
                                        : 1.0;
    levels_max += s.quench ? 1.0 : 0.0;
    run->sweep_cap = (int64_t)(levels_max * (double)(s.fixed_sweeps > 0 ? s.fixed_sweeps : s.k_max)) + 1;
    run->batch = 1;
    run->done_sweeps = 0;
    return tc_plan(c, run, R, R);
}

// One sweep as direct launches; with `timed`, event pairs bracket each GEMM.
// With the overlap, panel p's GEMM (on the side stream) leaves panel p-1's
// K range out and waits only for chain p-2, whose G buffer it overwrites;
// chain p waits for GEMM p and takes panel p-1's part of its fields from
// chain p-1 (Gx).
int tc_enqueue_sweep(mars_ctx* c, TcRun* run, cudaStream_t st, bool timed)
{
    const bool ov = run->overlap;
    const int P = run->P;
    if (timed) run->timed_rows.clear();
    // the chains cover the slots below the active prefix the plan was made for
    TcState tc = run->t;
    tc.R = run->chain_slots;
    if (run->pair) {
        // panels in pairs: one GEMM for panels pp and pp+1, chain pp (which
        // adds its new spins to panel pp+1's fields), chain pp+1
        const int kb_per_panel = run->g.fp8 ? 1 : 2;
        for (int pp = 0; pp < P; pp += 2) {
            const int e = (int)run->timed_rows.size();
            TcPanel g = run->g;
            g.p0 = pp * 128;
            g.G = run->Gbuf[0];
            const bool two = pp + 1 < P;
            if (timed) MARS_CUDA(c, cudaEventRecord(c->prof[2 * e], st));
            if (two) {
                g.G1 = run->Gbuf[1];
                g.skip_kb = kb_per_panel * pp;
                MARS_CUDA(c, launch_tc_pair_gemm(run->tmJ, run->tmS, g, run->gemm_tiles, run->splitk, st));
            } else {
                g.skip_kb = -1;
                MARS_CUDA(c, launch_tc_panel_gemm(run->tmJ, run->tmS, g, kTcBN, run->gemm_tiles, run->splitk, st));
            }
            if (timed) {
                MARS_CUDA(c, cudaEventRecord(c->prof[2 * e + 1], st));
                run->timed_rows.push_back(two ? 256 : 128);
            }
            // chain pp's fields come from the GEMM just before it; chain pp+1's
            // from the same GEMM, two kernels back
            MARS_CUDA(c, launch_tc_chain(tc, pp, run->rpw, run->chain_warps, run->Gbuf[0], nullptr, two ? run->Gx[0] : nullptr,
                                         false, st));
            if (two)
                MARS_CUDA(c, launch_tc_chain(tc, pp + 1, run->rpw, run->chain_warps, run->Gbuf[1], run->Gx[0], nullptr, true, st));
        }
        MARS_CUDA(c, launch_tc_advance(run->t, st));
        return MARS_OK;
    }
    cudaStream_t gs = ov ? run->side : st;
    if (ov) {
        MARS_CUDA(c, cudaEventRecord(run->ev[0], st));
        MARS_CUDA(c, cudaStreamWaitEvent(gs, run->ev[0], 0));
    }
    for (int pp = 0; pp < P; ++pp) {
        TcPanel g = run->g;
        g.p0 = pp * 128;
        g.G = run->Gbuf[pp & 1];
        g.skip_kb = ov && pp > 0 ? (g.fp8 ? 1 : 2) * (pp - 1) : -1;  // panel pp-1's K blocks
        if (ov && pp >= 2) MARS_CUDA(c, cudaStreamWaitEvent(gs, run->ev[2 + 2 * (pp - 2)], 0));
        if (timed) MARS_CUDA(c, cudaEventRecord(c->prof[2 * pp], gs));
        MARS_CUDA(c, launch_tc_panel_gemm(run->tmJ, run->tmS, g, kTcBN, run->gemm_tiles, run->splitk, gs));
        if (timed) {
            MARS_CUDA(c, cudaEventRecord(c->prof[2 * pp + 1], gs));
            run->timed_rows.push_back(128);
        }
        if (ov) {
            MARS_CUDA(c, cudaEventRecord(run->ev[1 + 2 * pp], gs));
            MARS_CUDA(c, cudaStreamWaitEvent(st, run->ev[1 + 2 * pp], 0));
        }
        const float* gx_in = ov && pp > 0 ? run->Gx[pp & 1] : nullptr;
        float* gx_out = ov && pp + 1 < P ? run->Gx[(pp + 1) & 1] : nullptr;
        // the GEMM's event edge into the chain may be captured as a
        // programmatic edge too, so its fields are read after the wait
        MARS_CUDA(c, launch_tc_chain(tc, pp, run->rpw, run->chain_warps, run->Gbuf[pp & 1], gx_in, gx_out, false, st));
        if (ov) MARS_CUDA(c, cudaEventRecord(run->ev[2 + 2 * pp], st));
    }
    MARS_CUDA(c, launch_tc_advance(run->t, st));
    return MARS_OK;
}

// Enqueue run->batch sweeps (the first one with timed GEMMs when profiling,
// the rest as replays of the captured sweep), then the copy of the counters
// to pinned memory.
int tc_enqueue_batch(mars_ctx* c, TcRun* run, cudaStream_t st)
{
    int rc;
    // Finished replicas below the active prefix: move the active ones to the
    // front (a replica's arithmetic does not depend on its slot).
    if (run->compact && run->h_counters && run->h_counters[1] > 0 &&
        run->h_counters[0] - run->h_counters[1] >= 16) {
        MARS_CUDA(c, launch_tc_compact(run->t, run->rep_mut, run->cp, run->h_counters[0], st));
        run->h_counters[0] = run->h_counters[1];
        run->compactions += 1;
    }
    if (run->active_at_batch > 0 &&
        (rc = tc_plan(c, run, run->active_at_batch, run->h_counters ? run->h_counters[0] : run->t.R)))
        return rc;
    if (run->profile) {
        while ((int)c->prof.size() < 2 * run->P) {
            cudaEvent_t e;
            MARS_CUDA(c, cudaEventCreate(&e));
            c->prof.push_back(e);
        }
    }
    if (run->persist) {
        // one cooperative launch for the whole batch, then the active prefix
        TcPersist q = run->pp;
        q.sweeps = run->batch;
        MARS_CUDA(c, cudaMemsetAsync(run->flags, 0, (2 * (size_t)kTcMaxBatch * run->P + 1) * sizeof(int32_t), st));
        MARS_CUDA(c, launch_tc_sweeps(run->tmJ, run->tmS, run->t, run->g, q, run->rpw, st));
        MARS_CUDA(c, launch_tc_prefix(run->t, st));
        run->timed_rows.clear();
        run->done_sweeps += run->batch;
        MARS_CUDA(c, cudaMemcpyAsync(run->h_counters, run->t.counters, 4 * sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, st));
        return MARS_OK;
    }
    for (int b = 0; b < run->batch; ++b) {
        if (b == 0 && run->profile) {
            if ((rc = tc_enqueue_sweep(c, run, st, true))) return rc;
            continue;
        }
        if (!run->exec) {
            MARS_CUDA(c, cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
            rc = tc_enqueue_sweep(c, run, st, false);
            cudaGraph_t graph = nullptr;
            const cudaError_t e = cudaStreamEndCapture(st, &graph);
            if (rc) return rc;
            if (e != cudaSuccess) return fail(c, MARS_EDEVICE, "sweep capture failed: %s", cudaGetErrorString(e));
            run->graph = graph;
            MARS_CUDA(c, cudaGraphInstantiate(&run->exec, run->graph, 0));
        }
        MARS_CUDA(c, cudaGraphLaunch(run->exec, st));
    }
    run->done_sweeps += run->batch;
    MARS_CUDA(c, cudaMemcpyAsync(run->h_counters, run->t.counters, 4 * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, st));
    return MARS_OK;
}

// After a batch's counters arrived: 1 = more sweeps needed, 0 = done, < 0 = error.
int tc_after_batch(mars_ctx* c, TcRun* run)
{
    if (run->h_counters[2] != 0) return fail(c, MARS_ETIMEOUT, "a tensor-core pipeline wait gave up");
    if (run->h_counters[1] == 0) return 0;
    if (run->done_sweeps > run->sweep_cap) return fail(c, MARS_EDEVICE, "descent exceeded its sweep bound");
    run->active_at_batch = run->h_counters[1];
    run->batch = std::min(run->batch * 2, kTcMaxBatch);
    return 1;
}

// The dense descent on tensor cores, blocking: slots in start-temperature
// order, a sweep = for each 128-spin panel {BF16 panel GEMM, in-panel
// sequential chain}, then the level step; the host checks the active count
// between batches of sweeps.
int run_dense_tc(mars_ctx* c, Instance* in, const mars_params* p, const DevSolve& s,
                 const std::vector<int32_t>& reps, float t0_max, Scratch& S, TcProfile* prof,
                 bool polish)
{
    (void)p;
    cudaStream_t st = c->stream;
    int rc;
    int32_t* rep = nullptr;
    if ((rc = S.get(s.R, &rep))) return rc;
    MARS_CUDA(c, cudaMemcpyAsync(rep, reps.data(), s.R * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    TcRun run;
    // A blocking solve may run its partly active batches as one cooperative
    // launch each (MARS_TC_PERSIST=1; off by default: on a GB300 at N = 8192
    // it measured slower than the launched overlap, 1.38 against 0.76 ms per
    // sweep with 128 replicas active); served requests share the device with
    // other requests' kernels, which could keep such a launch from being
    // resident at once, and never use it.
    run.allow_persist = env_flag("MARS_TC_PERSIST", 0) != 0;
    auto get = [&](size_t bytes, void** out) -> int {
        unsigned char* q = nullptr;
        int r = S.get(bytes, &q);
        *out = q;
        return r;
    };
    if ((rc = tc_setup(c, in->dev, s, rep, t0_max, p->precision == MARS_FP8, st, get, &run))) return rc;
    prof->launches += 2;  // start states, active prefix
    // The compaction's scratch (a copy of the per-slot arrays) is taken only
    // when it fits in half of the free device memory and of what the budget
    // has left; otherwise the solve runs without compaction.
    const size_t cp_rows = (size_t)s.R * run.t.n_pad;
    const size_t cp_bytes = cp_rows * (sizeof(float) + (run.t.S8 ? 1 : sizeof(__nv_bfloat16))) +
                            (size_t)s.R * (sizeof(double) + 2 * sizeof(float) + 7 * sizeof(int32_t));
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const bool cp_fits = 2 * cp_bytes <= free_b && (!c->budget || c->used + 2 * cp_bytes <= c->budget);
    if (env_flag("MARS_TC_COMPACT", 1) != 0 && s.R > kTcBN && cp_fits) {
        const size_t R = (size_t)s.R, rows = cp_rows;
        TcCompact& cp = run.cp;
        if ((rc = S.get(R, &cp.perm)) || (rc = S.get(rows, &cp.S)) ||
            (run.t.S8 ? (rc = S.get(rows, &cp.S8)) : (rc = S.get(rows, &cp.Sb))) || (rc = S.get(R, &cp.T)) ||
            (rc = S.get(R, &cp.invT)) || (rc = S.get(R, &cp.d)) || (rc = S.get(R, &cp.active)) ||
            (rc = S.get(R, &cp.levels)) || (rc = S.get(R, &cp.lvl_sweeps)) || (rc = S.get(R, &cp.sweeps)) ||
            (rc = S.get(R, &cp.capped)) || (rc = S.get(R, &cp.rep)))
            return rc;
        run.compact = true;
        run.rep_mut = rep;
    }
    int32_t* pinned = nullptr;
    MARS_CUDA(c, cudaMallocHost((void**)&pinned, 4 * sizeof(int32_t)));
    run.h_counters = pinned;
    run.profile = true;
    MARS_CUDA(c, cudaMemcpyAsync(run.h_counters, run.t.counters, 4 * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, st));
    cudaError_t se = cudaStreamSynchronize(st);
    run.active_at_batch = run.h_counters[1];
    int state = se == cudaSuccess ? (run.h_counters[1] > 0 ? 1 : 0) : -1;
    int64_t compactions_seen = 0;
    while (state == 1) {
        const int32_t active_now = run.active_at_batch;
        if ((rc = tc_enqueue_batch(c, &run, st))) { cudaFreeHost(pinned); return rc; }
        // per sweep: the GEMMs (one per panel, or per pair), P chains, the level step and
        // prefix; a persistent batch is one kernel and the prefix
        const int gemms = run.pair ? (run.P + 1) / 2 : run.P;
        prof->launches += run.persist ? 2 : (int64_t)run.batch * (gemms + run.P + 2);
        prof->launches += 2 * (run.compactions - compactions_seen);  // order and gather
        compactions_seen = run.compactions;
        se = cudaStreamSynchronize(st);
        if (se != cudaSuccess) break;
        for (size_t e = 0; e < run.timed_rows.size(); ++e) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, c->prof[2 * e], c->prof[2 * e + 1]);
            prof->gemm_seconds += ms * 1e-3;
            prof->gemm_launches += 1;
            prof->gemm_flops += 2.0 * run.timed_rows[e] * (double)in->dev.n * (double)active_now;
        }
        run.timed_rows.clear();
        state = tc_after_batch(c, &run);
    }
    cudaFreeHost(pinned);
    if (se != cudaSuccess) return fail(c, MARS_EDEVICE, "CUDA error: %s", cudaGetErrorString(se));
    if (state < 0) return state;
    if (!polish) MARS_CUDA(c, cudaEventRecord(c->ev3, st));
    MARS_CUDA(c, launch_tc_finalize(run.t, in->dev, s, st));
    prof->launches += 1;
    if (polish) {
        // FP32 polish: the SIMT dense path re-converges each replica's last
        // level from its BF16 final state; it writes the spins and energies.
        float* m_out = nullptr;
        double* t_last = nullptr;
        if ((rc = S.get((size_t)s.R * in->dev.n, &m_out))) return rc;
        if ((rc = S.get(s.R, &t_last))) return rc;
        MARS_CUDA(c, launch_tc_export(run.t, in->dev, m_out, t_last, st));
        DevSolve ps = s;
        ps.m0 = m_out;
        ps.t_first = t_last;
        ps.one_level = 1;
        ps.add_counts = 1;
        ps.jacobi = 0;
        DensePlan dp = plan_dense(in->dev, s.R, 0, c->device);
        if (dp.scratch_floats && (rc = S.get(dp.scratch_floats, &ps.m_scratch))) return rc;
        MARS_CUDA(c, launch_dense(in->dev, ps, dp, st));
        MARS_CUDA(c, cudaEventRecord(c->ev3, st));
        prof->launches += 2;
    }
    return MARS_OK;
}

