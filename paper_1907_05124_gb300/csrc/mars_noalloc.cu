// mars_solve_noalloc: mars_solve with every per-solve buffer in one static
// device array, for callers that cannot allocate device memory while they
// run. The paper has no counterpart to this entry point.
//
// The static array g_noalloc_scratch below is MARS_NOALLOC_SCRATCH_BYTES
// (16 MiB) of __device__ memory that every GPU which loads this library's
// module keeps until the process exits. Host code never names it directly:
// its device address comes from cudaGetSymbolAddress, taken on a context's
// first call (with the context's device current) and cached in the context.
#include "../../include/mars.h"
#include "mars_internal.h"

#include <cmath>
#include <cstring>

namespace mars {
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MARS_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device, looked up once
// per context and cached in it (*cache). A context lives on one device and
// its device memory does not survive a device reset, so neither does the
// cache: a caller that resets the device creates a new context, whose first
// call looks the address up again.
int scratch_address(void** cache, void** out)
{
    if (!*cache) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return MARS_EDEVICE;
        }
        *cache = p;
    }
    *out = *cache;
    return MARS_OK;
}

// Replicas in index order, then the work counter and status word at zero:
// the array keeps whatever the previous call left there.
__global__ void noalloc_prepare(int32_t* tile_rep, int32_t R, int32_t total, int32_t* counters)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        tile_rep[i] = i < R ? i : -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counters[0] = 0;
        counters[1] = 0;
    }
}

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace mars

using namespace mars;

extern "C" int mars_solve_noalloc(mars_ctx* c, int32_t id, const mars_params* p,
                                  int8_t* best_spins, double* energies, mars_result* result)
{
    if (!c || !p || !best_spins) return MARS_EINVAL;
    NoallocView v;
    int rc = noalloc_view(c, id, &v);
    if (rc) return rc;
    const DevInstance& in = *v.inst;
    const int32_t R = p->replicas, n = in.n;
    if (R < 1) return noalloc_fail(c, MARS_EINVAL, "replicas must be >= 1");
    if (!std::isfinite(p->t_min) || !std::isfinite(p->t_max) || p->t_min > p->t_max)
        return noalloc_fail(c, MARS_EINVAL, "need finite t_min <= t_max");
    if (!(p->c_step > 0.0) || !std::isfinite(p->c_step) || p->t_max / p->c_step > 1e6)
        return noalloc_fail(c, MARS_EINVAL, "need c_step > 0 and t_max / c_step <= 1e6");
    if (!(p->d_min >= 0.0) || p->k_max < 1 || p->fixed_sweeps < 0)
        return noalloc_fail(c, MARS_EINVAL, "need d_min >= 0, k_max >= 1, fixed_sweeps >= 0");
    if (p->update != MARS_UPDATE_GS || p->precision != MARS_FP32 || p->method != MARS_METHOD_MARS)
        return noalloc_fail(c, MARS_EINVAL, "mars_solve_noalloc runs sequential FP32 MARS sweeps only");
    if (p->schedule != MARS_SCHEDULE_LINEAR || p->quench)
        return noalloc_fail(c, MARS_EINVAL, "mars_solve_noalloc runs the paper's linear schedule only");
    if ((p->m0 || p->t0) && !(p->flags & MARS_DEVICE_PTR))
        return noalloc_fail(c, MARS_EINVAL, "m0/t0 must be device pointers (MARS_DEVICE_PTR)");
    if (p->t0)
        return noalloc_fail(c, MARS_EINVAL, "mars_solve_noalloc draws t0 itself (pass t0 = NULL)");

    // Launch plan: only plans that need no buffer beyond the static array.
    SparsePlan sp;
    DensePlan dp;
    int rt = 1;
    if (in.dense) {
        dp = plan_dense(in, R, 0, v.device);
        if (dp.scratch_floats) return noalloc_fail(c, MARS_EINVAL, "n too large for the on-chip dense path");
    } else {
        if (!plan_sparse_sell(in, R, v.device, &sp)) sp = plan_sparse(in, R, 0, v.device);
        if (sp.scratch_floats) return noalloc_fail(c, MARS_EINVAL, "n too large for the on-chip sparse path");
        rt = sp.rt;
    }
    const int32_t ntiles = (R + rt - 1) / rt;

    // Layout of the static array; every piece starts on a 256-byte boundary.
    size_t off = 0;
    const size_t o_t0 = off;      off = round_up(off + (size_t)R * sizeof(float));
    const size_t o_tiles = off;   off = round_up(off + (size_t)ntiles * rt * sizeof(int32_t));
    const size_t o_count = off;   off = round_up(off + 2 * sizeof(int32_t));
    const size_t o_e = off;       off = round_up(off + (size_t)R * sizeof(double));
    const size_t o_ei = off;      off = round_up(off + (size_t)R * sizeof(long long));
    const size_t o_sw = off;      off = round_up(off + (size_t)R * sizeof(int32_t));
    const size_t o_lv = off;      off = round_up(off + (size_t)R * sizeof(int32_t));
    const size_t o_cp = off;      off = round_up(off + (size_t)R * sizeof(int32_t));
    const size_t o_res = off;     off = round_up(off + sizeof(DevResult));
    const size_t o_sigma = off;   off = round_up(off + (size_t)R * n);
    if (off > (size_t)MARS_NOALLOC_SCRATCH_BYTES)
        return noalloc_fail(c, MARS_EINVAL,
                            "replicas * n needs %zu bytes of scratch; the static limit is %zu",
                            off, (size_t)MARS_NOALLOC_SCRATCH_BYTES);

    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != v.device) cudaSetDevice(v.device);
    unsigned char* base = nullptr;
    rc = scratch_address(v.scratch_base, (void**)&base);
    if (rc) {
        if (prev >= 0 && prev != v.device) cudaSetDevice(prev);
        return noalloc_fail(c, rc, "cudaGetSymbolAddress of the static scratch failed");
    }
    cudaStream_t st = v.stream;
    DevSolve s;
    s.R = R;
    s.seed = p->seed;
    s.stream = p->stream;
    s.c_step = p->c_step;
    s.d_min = (float)p->d_min;
    s.k_max = p->k_max;
    s.fixed_sweeps = p->fixed_sweeps;
    s.jacobi = 0;
    s.m0 = p->m0;
    s.t0 = (const float*)(base + o_t0);
    s.tile_rep = (const int32_t*)(base + o_tiles);
    s.work_counter = (int32_t*)(base + o_count);
    s.status = s.work_counter + 1;
    s.energy = (double*)(base + o_e);
    s.energy_i64 = (long long*)(base + o_ei);
    s.sweeps = (int32_t*)(base + o_sw);
    s.levels = (int32_t*)(base + o_lv);
    s.capped = (int32_t*)(base + o_cp);
    s.sigma = (int8_t*)(base + o_sigma);
    s.ntiles = ntiles;
    s.rt = rt;
    DevResult* dres = (DevResult*)(base + o_res);

    cudaError_t e = launch_draw(p->seed, p->stream, 0, R, 0, p->t_min, p->t_max, nullptr,
                                (float*)(base + o_t0), st);
    if (e == cudaSuccess) {
        noalloc_prepare<<<(ntiles * rt + 255) / 256, 256, 0, st>>>((int32_t*)(base + o_tiles), R,
                                                                 ntiles * rt, s.work_counter);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = in.dense ? launch_dense(in, s, dp, st)
                     : (sp.sell ? launch_sparse_sell(in, s, sp, st) : launch_sparse(in, s, sp, st));
    if (e == cudaSuccess) e = launch_best(s, n, in.integer, best_spins, dres, st);
    if (e == cudaSuccess && energies)
        e = cudaMemcpyAsync(energies, s.energy, (size_t)R * sizeof(double), cudaMemcpyDeviceToDevice, st);
    DevResult hres;
    int32_t hstatus = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hres, dres, sizeof hres, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hstatus, s.status, sizeof hstatus, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (prev >= 0 && prev != v.device) cudaSetDevice(prev);
    if (e != cudaSuccess) return noalloc_fail(c, MARS_EDEVICE, "CUDA error: %s", cudaGetErrorString(e));
    if (hstatus != kDevOk) return noalloc_fail(c, MARS_EDEVICE, "device status %d", hstatus);
    if (result) {
        std::memset(result, 0, sizeof *result);
        result->best_energy = hres.best_energy;
        result->best_energy_i64 = hres.best_energy_i64;
        result->best_cut = (v.total_weight - hres.best_energy) / 2.0;
        result->best_replica = hres.best_replica;
        result->hits = hres.hits;
        result->mean_energy = hres.sum_energy / R;
        result->sweeps = hres.sweeps;
        result->spin_updates = hres.sweeps * (int64_t)n;
        result->levels = hres.levels;
        result->capped_levels = hres.capped;
        result->integer = in.integer;
        result->energy_err_bound = v.energy_err_bound;
        result->status = MARS_OK;
    }
    return MARS_OK;
}
