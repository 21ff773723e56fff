// Sparse MARS descent, fast path: sliced-ELL couplings and on-chip replicas.
//
// Same method and same schedule as kernels_sparse.cu (Section 3, Algorithm 1:
// sequential sweeps reproduced level by level), with a layout built for the
// SM instead of a plain CSR walk:
//
//  * Within a level the runtime sorts spins by degree and cuts them into
//    slices of 32 consecutive new labels (any order inside a level gives the
//    sequential sweep's values, since those spins share no coupling). A
//    slice's couplings are stored slot-major, padded to the slice's largest
//    degree: entry d of row q sits at off + 32*d + q. A warp walks one slice,
//    lane q owns row q, and each of its loads is one coalesced 128-byte line.
//    Padding points at a dummy spin whose magnetisation is held at 0.
//  * +-1 couplings are one 32-bit word: column | sign bit. General weights
//    are a (column, value) pair.
//  * A thread owns one spin for all RT replicas of the tile: one coupling
//    load, one RT-wide shared-memory gather, RT multiply-adds.
//
// The tile's magnetisations m[i*RT + k] live in shared memory for the whole
// descent; the dummy row n is zero. Only the sweeps' parallel steps need a
// block barrier. When not even one replica's m fits on chip, the same job
// runs with m in a global-memory slab per CTA (kernels_sparse_slab.cu).
#include "sell_job.cuh"

#include <algorithm>
#include <cstdlib>

namespace mars {
namespace {

template <int RT, int NT, int FMT, int DEG>
__global__ void __launch_bounds__(NT, 1024 / NT) sparse_sell_kernel(DevInstance in, DevSolve s)
{
    extern __shared__ __align__(16) float m[];  // (n+1)*RT, then the staged table (FMT 2)
    __shared__ SlotState<RT, NT / 32> S;
    run_job<RT, NT, FMT, DEG>(in, s, m, S);
}

// Several instances in one persistent launch: CTAs work through the job list
// in order, each draining one instance's replica queue before it moves on, so
// instances of uneven size and replica count share the SMs without a launch
// per instance. The coupling format is chosen per job.
// One job of a batched launch with its own slot width (1 or 2, job.rt) and
// coupling format under the CTA's two-slot bookkeeping.
template <int NT>
__device__ void run_batch_job(const BatchJob& job, float* m, SlotState<2, NT / 32>& S)
{
    switch (job.rt * 4 + job.fmt) {
    case 4 + 3: run_job<1, NT, 3, 0, 2>(job.in, job.s, m, S); break;
    case 4 + 2: run_job<1, NT, 2, 0, 2>(job.in, job.s, m, S); break;
    case 4 + 1: run_job<1, NT, 1, 0, 2>(job.in, job.s, m, S); break;
    case 4 + 0: run_job<1, NT, 0, 0, 2>(job.in, job.s, m, S); break;
    case 8 + 3: run_job<2, NT, 3, 0, 2>(job.in, job.s, m, S); break;
    case 8 + 2: run_job<2, NT, 2, 0, 2>(job.in, job.s, m, S); break;
    case 8 + 1: run_job<2, NT, 1, 0, 2>(job.in, job.s, m, S); break;
    default: run_job<2, NT, 0, 0, 2>(job.in, job.s, m, S); break;
    }
}

// Several instances in one persistent launch: CTAs work through the job list
// in order, each job's replica queue drained by every CTA before it moves on
// (a job is a CTA's current work until its queue is empty). Shared memory is
// sized for the most demanding job; slot width and coupling format are chosen
// per job.
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) sparse_sell_batch_kernel(const BatchJob* jobs, int njobs,
                                                                       int* cursor)
{
    extern __shared__ __align__(16) float m[];
    __shared__ SlotState<2, NT / 32> S;
    __shared__ BatchJob s_jobcopy;  // the current job's descriptors, read from shared memory
    __shared__ int s_job;
    for (;;) {
        if (threadIdx.x == 0) {
            int j = *((volatile int*)cursor);
            while (j < njobs && *((volatile int*)jobs[j].s.work_counter) >= jobs[j].s.R) {
                atomicMax(cursor, j + 1);
                ++j;
            }
            s_job = j < njobs ? j : -1;
        }
        __syncthreads();
        const int j = s_job;
        if (j < 0) break;
        {
            const int* src = reinterpret_cast<const int*>(jobs + j);
            int* dst = reinterpret_cast<int*>(&s_jobcopy);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchJob) / sizeof(int)); w += blockDim.x)
                dst[w] = src[w];
        }
        __syncthreads();
        run_batch_job<NT>(s_jobcopy, m, S);
        __syncthreads();
    }
}

// Persistent serving kernel: CTAs take replicas from the jobs published in the
// ring, oldest first; when none is left, thread 0 polls the ring's tail
// (about 2 us apart, at most idle_polls times) and the CTA exits when nothing
// new arrives. Descriptors written by the host's copies are read through
// volatile loads (past L1), after the tail that published them.
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) serve_ring_kernel(ServeRing* ring, int idle_polls)
{
    extern __shared__ __align__(16) float m[];
    __shared__ SlotState<2, NT / 32> S;
    __shared__ BatchJob s_jobcopy;
    __shared__ int s_job;
    for (;;) {
        if (threadIdx.x == 0) {
            int found = -1;
            for (int poll = 0; poll <= idle_polls; ++poll) {
                int c = *reinterpret_cast<volatile int*>(&ring->cursor);
                const int tail = *reinterpret_cast<volatile int*>(&ring->tail);
                __threadfence();
                while (c < tail) {
                    const int k = c % kRingCap;
                    const int taken = *reinterpret_cast<volatile int*>(&ring->slots[k].taken);
                    const int R = *reinterpret_cast<volatile int*>(&ring->jobs[k].s.R);
                    if (taken < R) break;
                    atomicMax(&ring->cursor, c + 1);
                    ++c;
                }
                if (c < tail) {
                    found = c;
                    break;
                }
                if (*reinterpret_cast<volatile int*>(&ring->stop)) break;
                __nanosleep(2000);
            }
            s_job = found;
        }
        __syncthreads();
        const int j = s_job;
        if (j < 0) break;
        {
            const volatile int* src = reinterpret_cast<const volatile int*>(ring->jobs + j % kRingCap);
            int* dst = reinterpret_cast<int*>(&s_jobcopy);
            for (int w = threadIdx.x; w < (int)(sizeof(BatchJob) / sizeof(int)); w += blockDim.x)
                dst[w] = src[w];
        }
        __syncthreads();
        run_batch_job<NT>(s_jobcopy, m, S);
        __syncthreads();
    }
}

template <int RT, int NT, int DEG>
const void* pick_nt(int fmt)
{
    return fmt == 3 ? (const void*)sparse_sell_kernel<RT, NT, 3, DEG>
         : fmt == 2 ? (const void*)sparse_sell_kernel<RT, NT, 2, DEG>
         : fmt == 1 ? (const void*)sparse_sell_kernel<RT, NT, 1, DEG>
                    : (const void*)sparse_sell_kernel<RT, NT, 0, DEG>;
}

// Regular instances of degree 4 or 6 (square and cubic lattices) get a fully
// unrolled coupling loop in the default 1024-thread shapes.
const void* pick(int rt, int nt, int fmt, int deg)
{
    if (nt == 1024 && (deg == 4 || deg == 6) && fmt != 0) {
        switch (rt) {
        case 1: return deg == 4 ? pick_nt<1, 1024, 4>(fmt) : pick_nt<1, 1024, 6>(fmt);
        case 2: return deg == 4 ? pick_nt<2, 1024, 4>(fmt) : pick_nt<2, 1024, 6>(fmt);
        case 4: return deg == 4 ? pick_nt<4, 1024, 4>(fmt) : pick_nt<4, 1024, 6>(fmt);
        }
    }
    if (nt == 512) {
        switch (rt) {
        case 1: return pick_nt<1, 512, 0>(fmt);
        case 2: return pick_nt<2, 512, 0>(fmt);
        case 4: return pick_nt<4, 512, 0>(fmt);
        }
    } else if (nt == 1024) {
        switch (rt) {
        case 1: return pick_nt<1, 1024, 0>(fmt);
        case 2: return pick_nt<2, 1024, 0>(fmt);
        case 4: return pick_nt<4, 1024, 0>(fmt);
        }
    }
    return nullptr;
}

int env_int(const char* name, int dflt)
{
    const char* v = std::getenv(name);
    return v && *v ? std::atoi(v) : dflt;
}

}  // namespace

// Launch shape: replica slots per CTA (RT) and threads per CTA. A GB300
// sweep of the six shapes on the 2-D L=100 lattice, R=1024 (spin-updates/s):
// RT=2 with 1024 threads 3.46e11; RT=1/1024 2.63e11; RT=4/1024 2.64e11;
// the 512-thread shapes 2.0-2.2e11. Wider CTAs give a lone replica's sweep
// more threads; two slots amortise the coupling loads without the 4-wide
// tail. The instance's launch shape (mars_autotune, mars_set_shape), else
// MARS_SELL_RT / MARS_SELL_THREADS / MARS_SELL_SMEM_TABLE, override it.
bool plan_sparse_sell(const DevInstance& in, int R, int device, SparsePlan* p)
{
    if (!in.slices || (!in.sell_pm1 && !in.sell_gen)) return false;
    int sms = 1, optin = 48 * 1024;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t budget = (size_t)optin - 12 * 1024;  // static shared memory and slack
    const LaunchShape& sh = in.shape;
    int rt = sh.sell_rt >= 0 ? sh.sell_rt : env_int("MARS_SELL_RT", 2);
    int nt = sh.sell_threads >= 0 ? sh.sell_threads : env_int("MARS_SELL_THREADS", 1024);
    const int smem_table = sh.sell_smem_table >= 0 ? sh.sell_smem_table : env_int("MARS_SELL_SMEM_TABLE", 1);
    if (rt != 1 && rt != 2 && rt != 4) rt = 1;
    if (nt != 512 && nt != 1024) nt = 512;
    auto m_bytes = [&](int c) { return align16((size_t)(in.n + 1) * c * sizeof(float)); };
    const size_t table = (size_t)in.nslices * 16 + (size_t)in.sell_len * 2;
    // Halfword couplings staged on chip when they fit beside the magnetisations.
    int fmt = in.sell_pm1 ? 1 : 0;
    if (in.sell16 && smem_table) {
        int c = rt;
        while (c > 1 && m_bytes(c) + table > budget) c /= 2;
        if (m_bytes(c) + table <= budget) {
            fmt = 2;
            rt = c;
        }
    }
    const int rt_asked = rt;
    if (fmt != 2) {
        while (rt > 1 && m_bytes(rt) > budget) rt /= 2;
        if (m_bytes(rt) > budget) {
            // Not even one replica fits on chip: per-CTA slabs of global
            // memory, the asked slot width, one 1024-thread CTA per SM.
            const int sfmt = in.sell_pm1 ? 1 : 0;
            const int sdeg = sfmt == 1 && env_int("MARS_SELL_UNROLL", 1) ? in.regular_deg : 0;
            const void* k = pick_sell_slab(rt_asked, sfmt, sdeg);
            if (!k) return false;
            int per_sm = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 1024, 0);
            p->rt = rt_asked;
            p->onchip = 0;
            p->threads = 1024;
            p->entry = sfmt;
            p->smem = 0;
            p->sell = 1;
            p->deg = sdeg;
            p->grid = std::max(1, std::min((R + rt_asked - 1) / rt_asked, sms * std::max(per_sm, 1)));
            p->scratch_floats = (size_t)p->grid * sell_slab_floats(in.n, rt_asked);
            return true;
        }
        if (in.sell16 && env_int("MARS_SELL_HALF_L1", 1)) fmt = 3;  // halfwords through L1
    }
    p->rt = rt;
    p->onchip = 1;
    p->threads = nt;
    p->entry = fmt;
    p->smem = m_bytes(rt) + (fmt == 2 ? table : 0);
    p->sell = 1;
    const int deg = env_int("MARS_SELL_UNROLL", 1) ? in.regular_deg : 0;
    p->deg = deg;
    const void* k = pick(rt, nt, fmt, deg);
    if (!k) return false;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, p->smem);
    if (per_sm < 1) per_sm = 1;
    const int ntiles = (R + rt - 1) / rt;
    p->grid = std::max(1, std::min(ntiles, sms * per_sm));
    p->scratch_floats = 0;
    return true;
}

cudaError_t launch_sparse_sell(const DevInstance& in, const DevSolve& s, const SparsePlan& p,
                               cudaStream_t st)
{
    const void* k = p.onchip ? pick(p.rt, p.threads, p.entry, p.deg) : pick_sell_slab(p.rt, p.entry, p.deg);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    DevInstance a = in;
    DevSolve b = s;
    void* args[] = {&a, &b};
    return cudaLaunchKernel(k, dim3(p.grid), dim3(p.threads), args, p.smem, st);
}

namespace {
const void* pick_batch(int nt)
{
    return nt == 1024 ? (const void*)sparse_sell_batch_kernel<1024> : (const void*)sparse_sell_batch_kernel<512>;
}
}  // namespace

// Launch shape of a batch: per job the widest slot width (2, else 1) whose
// magnetisations fit on chip and its coupling format; shared memory of the
// most demanding job.
bool plan_sparse_batch(const DevInstance* ins, int count, int device, BatchPlan* p, int* fmts, int* rts)
{
    int sms = 1, optin = 48 * 1024;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t budget = (size_t)optin - 16 * 1024;
    const int rt_max = env_int("MARS_SELL_RT", 2) >= 2 ? 2 : 1;
    int nt = env_int("MARS_SELL_THREADS", 1024);
    if (nt != 512 && nt != 1024) nt = 1024;
    auto m_bytes = [&](int n, int c) { return align16((size_t)(n + 1) * c * sizeof(float)); };
    size_t smem = 0;
    for (int j = 0; j < count; ++j) {
        const DevInstance& in = ins[j];
        if (in.dense || !in.slices || (!in.sell_pm1 && !in.sell_gen)) return false;
        int rt = rt_max;
        while (rt > 1 && m_bytes(in.n, rt) > budget) rt /= 2;
        if (m_bytes(in.n, rt) > budget) return false;
        const size_t table = (size_t)in.nslices * 16 + (size_t)in.sell_len * 2;
        int fmt = in.sell_pm1 ? 1 : 0;
        if (in.sell16) fmt = 3;
        if (in.sell16 && env_int("MARS_SELL_SMEM_TABLE", 1) && m_bytes(in.n, rt) + table <= budget) fmt = 2;
        fmts[j] = fmt;
        rts[j] = rt;
        smem = std::max(smem, m_bytes(in.n, rt) + (fmt == 2 ? table : 0));
    }
    p->rt = 2;
    p->threads = nt;
    p->smem = smem;
    const void* k = pick_batch(nt);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, smem);
    p->grid = sms * std::max(per_sm, 1);
    return true;
}

cudaError_t launch_sparse_batch(const BatchJob* jobs, int count, int* cursor, const BatchPlan& p,
                                cudaStream_t st)
{
    const void* k = pick_batch(p.threads);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&jobs, (void*)&count, (void*)&cursor};
    return cudaLaunchKernel(k, dim3(p.grid), dim3(p.threads), args, p.smem, st);
}

bool plan_serve_ring(int device, RingPlan* p)
{
    int sms = 1, optin = 48 * 1024;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    p->rt = 2;
    p->threads = 1024;
    p->smem = (size_t)optin - 16 * 1024;  // static shared memory and slack
    const void* k = (const void*)serve_ring_kernel<1024>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem) != cudaSuccess)
        return false;
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, p->threads, p->smem);
    p->grid = sms * std::max(per_sm, 1);
    return true;
}

int ring_job_format(const DevInstance& in, const RingPlan& p, int* rt)
{
    if (in.dense || !in.slices || (!in.sell_pm1 && !in.sell_gen)) return -1;
    auto m_bytes = [&](int c) { return align16((size_t)(in.n + 1) * c * sizeof(float)); };
    *rt = m_bytes(2) <= p.smem ? 2 : 1;
    const size_t mb = m_bytes(*rt);
    if (mb > p.smem) return -1;
    const size_t table = (size_t)in.nslices * 16 + (size_t)in.sell_len * 2;
    if (in.sell16 && mb + table <= p.smem) return 2;
    if (in.sell16) return 3;
    return in.sell_pm1 ? 1 : 0;
}

cudaError_t launch_serve_ring(ServeRing* ring, const RingPlan& p, int idle_polls, cudaStream_t st)
{
    if (p.threads != 1024) return cudaErrorInvalidValue;
    const void* k = (const void*)serve_ring_kernel<1024>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&ring, (void*)&idle_polls};
    return cudaLaunchKernel(k, dim3(p.grid), dim3(p.threads), args, p.smem, st);
}

}  // namespace mars
