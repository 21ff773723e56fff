// Sparse MARS descent (Section 3, Algorithm 1) for CSR couplings.
//
// One CTA owns a tile of RT replicas and carries them through the whole
// descent: every level of temperature, every sweep, then sign-rounding and the
// exact energy. Replicas never interact, so a CTA needs no other CTA and there
// is no grid-wide barrier; CTAs take tiles from a global counter.
//
// A sweep visits spins in the instance's order, each update using the newest
// values (Gauss-Seidel). The runtime relabels spins by "level": a spin's level
// is one more than the deepest level among its neighbours visited before it.
// Spins of one level have no coupling between them, so a level is updated in
// parallel and gives exactly the values of the sequential sweep. A colour order
// has as many levels as colours (2 for an even periodic lattice).
//
// Layout: the tile's magnetisations are m[i*RT + k] (spin-major, RT replicas
// contiguous), in shared memory when n*RT*4 bytes fit, else in a per-CTA slab
// of global memory. Thread t always serves replica slot k = t % RT, so the
// per-replica running max d and the per-replica state live in registers and a
// handful of shared words.
#include "device_common.cuh"
#include "schedule.cuh"
#include "mars_internal.h"

#include <algorithm>

namespace mars {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

template <int RT, bool ONCHIP, bool JACOBI>
__global__ void __launch_bounds__(kThreads) sparse_descent_kernel(DevInstance in, DevSolve s)
{
    extern __shared__ __align__(16) float smem_m[];
    __shared__ double s_T[RT];
    __shared__ float s_invT[RT];
    __shared__ int s_lvl_sweeps[RT], s_sweeps[RT], s_levels[RT], s_capped[RT], s_active[RT];
    __shared__ float s_dred[kWarps][RT];
    __shared__ long long s_ei[kWarps][RT];
    __shared__ double s_ef[kWarps][RT];
    __shared__ int s_tile, s_any;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = tid % RT;
    const int n = in.n;
    const int nrt = n * RT;
    float* m = ONCHIP ? smem_m : s.m_scratch + (size_t)blockIdx.x * nrt;
    float* mnext = JACOBI ? s.m_next + (size_t)blockIdx.x * nrt : nullptr;

    for (;;) {
        if (tid == 0) s_tile = atomicAdd(s.work_counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= s.ntiles) break;
        const int r = s.tile_rep[tile * RT + k];

        // ---- start state: caller m0 or the counter-based draw -----------------
        for (int idx = tid; idx < nrt; idx += kThreads) {
            const int o = __ldg(in.new2old + idx / RT);
            float v = 0.f;
            if (r >= 0) v = s.m0 ? __ldg(s.m0 + (size_t)r * n + o) : draw_m0(s.seed, s.stream, r, o);
            m[idx] = v;
        }
        if (tid < RT) {
            // the first level (schedule.cuh)
            double T = 0.0;
            const bool act = r >= 0 && sched_first(s, (double)s.t0[r], &T);
            s_T[tid] = T;
            s_invT[tid] = act ? sched_inv_t(T) : 0.f;
            s_active[tid] = act;
            s_levels[tid] = act ? 1 : 0;
            s_lvl_sweeps[tid] = 0;
            s_sweeps[tid] = 0;
            s_capped[tid] = 0;
        }
        __syncthreads();

        // ---- levels of temperature and sweeps ---------------------------------
        for (;;) {
            if (tid == 0) {
                int any = 0;
#pragma unroll
                for (int q = 0; q < RT; ++q) any |= s_active[q];
                s_any = any;
            }
            __syncthreads();
            if (!s_any) break;
            const bool act = s_active[k] != 0;
            const float invT = s_invT[k];
            float dloc = 0.f;
            const int nlev = JACOBI ? 1 : in.nlev;
            for (int l = 0; l < nlev; ++l) {
                const int a0 = JACOBI ? 0 : __ldg(in.lvl_start + l) * RT;
                const int a1 = JACOBI ? nrt : __ldg(in.lvl_start + l + 1) * RT;
                if (act) {
                    for (int idx = a0 + tid; idx < a1; idx += kThreads) {
                        const int i = idx / RT;
                        const int e0 = __ldg(in.row_ptr + i), e1 = __ldg(in.row_ptr + i + 1);
                        float phi = 0.f;
                        for (int e = e0; e < e1; ++e)
                            phi = fmaf(__ldg(in.val + e), m[__ldg(in.col + e) * RT + k], phi);
                        if (in.h) phi += __ldg(in.h + i);
                        float sn;
                        if (JACOBI && s.nmfa) {
                            // noisy mean-field annealing: normalised field plus
                            // noise for iteration s_sweeps[k], then alpha-mixing
                            const float xi = s.nmfa_sigma > 0.f
                                                 ? nmfa_normal(s.seed, s.stream, (uint32_t)r,
                                                               (uint32_t)s_sweeps[k],
                                                               (uint32_t)__ldg(in.new2old + i))
                                                 : 0.f;
                            sn = nmfa_update(phi, __ldg(in.inv_norm + i), xi, s.nmfa_sigma, invT,
                                             s.nmfa_alpha, m[idx]);
                        } else {
                            sn = -tanhf(phi * invT);
                        }
                        dloc = fmaxf(dloc, fabsf(sn - m[idx]));
                        if (JACOBI) mnext[idx] = sn; else m[idx] = sn;
                    }
                }
                __syncthreads();
            }
            if (JACOBI) {
                if (act)
                    for (int idx = tid; idx < nrt; idx += kThreads) m[idx] = mnext[idx];
            }
            dloc = warp_reduce_strided<RT>(dloc, MaxOp());
            if (lane < RT) s_dred[warp][lane] = dloc;
            __syncthreads();
            if (tid < RT && s_active[tid]) {
                float d = 0.f;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) d = fmaxf(d, s_dred[w][tid]);
                int ls = s_lvl_sweeps[tid] + 1;
                s_sweeps[tid] += 1;
                double T = s_T[tid];
                const bool fixed = sched_fixed(s, T);
                const bool level_done = fixed ? ls >= s.fixed_sweeps : (d <= s.d_min || ls >= s.k_max);
                if (level_done) {
                    if (!fixed && !(d <= s.d_min)) s_capped[tid] += 1;
                    ls = 0;
                    if (sched_advance(s, &T)) {
                        s_T[tid] = T;
                        s_levels[tid] += 1;
                        s_invT[tid] = sched_inv_t(T);
                    } else {
                        s_active[tid] = 0;
                    }
                }
                s_lvl_sweeps[tid] = ls;
            }
            __syncthreads();
        }

        // ---- sign-round, outputs and exact energy ------------------------------
        long long ei = 0;
        double ef = 0.0;
        if (r >= 0) {
            for (int idx = tid; idx < nrt; idx += kThreads) {
                const int i = idx / RT;
                const float mv = m[idx];
                const int si = mv >= 0.f ? 1 : -1;
                const int o = __ldg(in.new2old + i);
                s.sigma[(size_t)r * n + o] = (int8_t)si;
                if (s.m_final) s.m_final[(size_t)r * n + o] = mv;
                const int e0 = __ldg(in.row_ptr + i), e1 = __ldg(in.row_ptr + i + 1);
                if (in.integer) {
                    int acc = 0;
                    for (int e = e0; e < e1; ++e) {
                        const int j = __ldg(in.col + e);
                        if (j > i) acc += (int)__ldg(in.val_i8 + e) * (m[j * RT + k] >= 0.f ? 1 : -1);
                    }
                    ei += (long long)(acc * si);
                    if (in.h) ei += (long long)__ldg(in.h + i) * si;
                } else {
                    double acc = 0.0;
                    for (int e = e0; e < e1; ++e) {
                        const int j = __ldg(in.col + e);
                        if (j > i) acc += __ldg(in.val_f64 + e) * (m[j * RT + k] >= 0.f ? 1.0 : -1.0);
                    }
                    ef += acc * si;
                    if (in.h_f64) ef += __ldg(in.h_f64 + i) * si;
                }
            }
        }
        ei = warp_reduce_strided<RT>(ei, SumOp());
        ef = warp_reduce_strided<RT>(ef, SumOp());
        if (lane < RT) { s_ei[warp][lane] = ei; s_ef[warp][lane] = ef; }
        __syncthreads();
        if (tid < RT && r >= 0) {
            long long ti = 0;
            double tf = 0.0;
            for (int w = 0; w < kWarps; ++w) { ti += s_ei[w][tid]; tf += s_ef[w][tid]; }
            s.energy[r] = in.integer ? (double)ti : tf;
            s.energy_i64[r] = in.integer ? ti : 0;
            s.sweeps[r] = s_sweeps[tid];
            s.levels[r] = s_levels[tid];
            s.capped[r] = s_capped[tid];
        }
        __syncthreads();
    }
}

template <int RT, bool ONCHIP, bool JACOBI>
const void* kernel_ptr()
{
    return (const void*)sparse_descent_kernel<RT, ONCHIP, JACOBI>;
}

const void* pick_kernel(int rt, bool onchip, bool jacobi)
{
#define MARS_PICK(R)                                                                 \
    if (rt == R) {                                                                    \
        if (onchip) return jacobi ? kernel_ptr<R, true, true>() : kernel_ptr<R, true, false>(); \
        return jacobi ? kernel_ptr<R, false, true>() : kernel_ptr<R, false, false>();           \
    }
    MARS_PICK(1)
    MARS_PICK(2)
    MARS_PICK(4)
    MARS_PICK(8)
#undef MARS_PICK
    return nullptr;
}

}  // namespace

SparsePlan plan_sparse(const DevInstance& in, int R, int jacobi, int device)
{
    int sms = 1, optin = 48 * 1024;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t budget = (size_t)optin - 8 * 1024;  // leave room for static shared memory
    SparsePlan p;
    p.threads = kThreads;
    // Largest tile that still gives every SM at least one tile and fits on chip.
    int rt = 0;
    for (int c : {8, 4, 2, 1}) {
        if ((size_t)in.n * c * sizeof(float) <= budget && (R + c - 1) / c >= std::min(R, sms)) {
            rt = c;
            break;
        }
    }
    if (rt == 0) {
        p.onchip = 0;
        rt = 1;
        for (int c : {8, 4, 2}) {
            if ((R + c - 1) / c >= std::min(R, sms)) { rt = c; break; }
        }
    }
    p.rt = rt;
    p.smem = p.onchip ? (size_t)in.n * rt * sizeof(float) : 0;
    const void* k = pick_kernel(rt, p.onchip != 0, jacobi != 0);
    if (p.smem > 48 * 1024)
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, p.smem);
    if (per_sm < 1) per_sm = 1;
    const int ntiles = (R + rt - 1) / rt;
    p.grid = std::max(1, std::min(ntiles, sms * per_sm));
    p.scratch_floats = (size_t)p.grid * in.n * rt * ((p.onchip ? 0 : 1) + (jacobi ? 1 : 0));
    return p;
}

cudaError_t launch_sparse(const DevInstance& in, const DevSolve& s, const SparsePlan& p,
                          cudaStream_t st)
{
    const void* k = pick_kernel(p.rt, p.onchip != 0, s.jacobi != 0);
    if (!k) return cudaErrorInvalidValue;
    if (p.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)p.smem);
        if (e != cudaSuccess) return e;
    }
    DevInstance a = in;
    DevSolve b = s;
    void* args[] = {&a, &b};
    return cudaLaunchKernel(k, dim3(p.grid), dim3(p.threads), args, p.smem, st);
}

}  // namespace mars
