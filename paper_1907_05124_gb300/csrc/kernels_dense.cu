// Dense MARS descent (Section 3, Algorithm 1) in FP32 on the SIMT cores.
//
// One warp carries one replica through the whole descent. A sweep visits the
// spins one after another (Gauss-Seidel: every spin shares a coupling with
// every other, so there is no parallelism inside one replica's sweep); the
// warp spreads each local field Phi_a = sum_b J_ab s_b over its 32 lanes and
// reduces it with shuffles, in compensated arithmetic (see Dot2). The
// replicas' magnetisations stay in shared memory. When n % 4 == 0 and a few
// rows fit beside them, the replicas of a CTA sweep in lockstep and each row
// of J is streamed into shared memory once per CTA by bulk copies
// (dense_staged_kernel); otherwise every warp reads J through the read-only
// cache. This is the plain FP32 path the tensor-core path is checked against.
#include "device_common.cuh"
#include "schedule.cuh"
#include "tc_primitives.cuh"
#include "mars_internal.h"

#include <algorithm>

namespace mars {
namespace {

constexpr int kDenseWarps = 4;
// Row buffers of the staged kernel (fewer when shared memory is short).
constexpr int kMaxStages = 4;

// Compensated dot product (Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, algorithm Dot2): every product's
// rounding error comes from an FMA, every sum's from TwoSum, and the errors
// are carried in a second float. The result is as accurate as a dot product
// evaluated in twice the working precision and then rounded, so the local
// field of a dense row does not lose ulps to a 32-lane tree of n terms.
// Explicit-rounding intrinsics keep the compiler from fusing the error terms.
struct Dot2 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_product(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);
        add_pair(p, pe);
    }
    __device__ __forceinline__ void add_pair(float v, float err)
    {
        const float t = __fadd_rn(s, v);
        const float z = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(v, z));
        s = t;
        c = __fadd_rn(c, __fadd_rn(e, err));
    }
    __device__ __forceinline__ float warp_total()
    {
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, s, m);
            const float c2 = __shfl_xor_sync(0xffffffffu, c, m);
            add_pair(s2, c2);
        }
        return __fadd_rn(s, c);
    }
};


template <bool LDG>
__device__ __forceinline__ float4 load4(const float4* p)
{
    if constexpr (LDG) return __ldg(p);
    return *p;
}

// Phi_a = sum_b J_ab m_b (+ h_a) of one row over the warp. Four Dot2 chains,
// one per float4 component, and two float4 loads per lane per step keep
// several loads in flight; the chains and then the lanes are merged with the
// same error-free additions, so the result keeps Dot2's accuracy. n4 = n / 4
// when the row and m are 16-byte aligned, else 0 (scalar loop). LDG: the row
// is in global memory (read-only path), else in shared memory.
template <bool LDG>
__device__ __forceinline__ float row_field(const float* __restrict__ Jrow, const float* m, int n,
                                           int n4, int lane, float h)
{
    Dot2 acc[4];
    const float4* J4 = reinterpret_cast<const float4*>(Jrow);
    const float4* m4 = reinterpret_cast<const float4*>(m);
    int k = lane;
#pragma unroll 2
    for (; k + 32 < n4; k += 64) {
        const float4 j0 = load4<LDG>(J4 + k), j1 = load4<LDG>(J4 + k + 32);
        const float4 x0 = m4[k], x1 = m4[k + 32];
        acc[0].add_product(j0.x, x0.x);
        acc[1].add_product(j0.y, x0.y);
        acc[2].add_product(j0.z, x0.z);
        acc[3].add_product(j0.w, x0.w);
        acc[0].add_product(j1.x, x1.x);
        acc[1].add_product(j1.y, x1.y);
        acc[2].add_product(j1.z, x1.z);
        acc[3].add_product(j1.w, x1.w);
    }
    if (k < n4) {
        const float4 j0 = load4<LDG>(J4 + k);
        const float4 x0 = m4[k];
        acc[0].add_product(j0.x, x0.x);
        acc[1].add_product(j0.y, x0.y);
        acc[2].add_product(j0.z, x0.z);
        acc[3].add_product(j0.w, x0.w);
    }
    for (int b = 4 * n4 + lane; b < n; b += 32)
        acc[0].add_product(LDG ? __ldg(Jrow + b) : Jrow[b], m[b]);
    acc[0].add_pair(h, 0.f);
    acc[0].add_pair(acc[1].s, acc[1].c);
    acc[2].add_pair(acc[3].s, acc[3].c);
    acc[0].add_pair(acc[2].s, acc[2].c);
    return acc[0].warp_total();
}

// One replica's place in the schedule (Algorithm 1's outer loop, schedule.cuh).
struct Level {
    double T = 0.0;
    float invT = 0.f;
    bool act = false;
    int levels = 0, sweeps = 0, capped = 0, lvl_sweeps = 0;

    // the first level, or the given one (the FP32 polish)
    __device__ void start(const DevSolve& s, int r)
    {
        if (s.t_first) {
            T = s.t_first[r];
            act = T > 0.0;
        } else {
            act = sched_first(s, (double)s.t0[r], &T);
        }
        invT = act ? sched_inv_t(T) : 0.f;
        levels = act ? 1 : 0;
    }
    // after a sweep whose largest change was d: stay, cool, or stop
    __device__ void after_sweep(const DevSolve& s, float d)
    {
        ++sweeps;
        ++lvl_sweeps;
        const bool fixed = sched_fixed(s, T);
        const bool level_done = fixed ? lvl_sweeps >= s.fixed_sweeps : (d <= s.d_min || lvl_sweeps >= s.k_max);
        if (!level_done) return;
        if (!fixed && !(d <= s.d_min)) ++capped;
        lvl_sweeps = 0;
        if (!s.one_level && sched_advance(s, &T)) {
            ++levels;
            invT = sched_inv_t(T);
        } else {
            act = false;
        }
    }
};

// Noisy mean-field annealing after a synchronous sweep that left the raw
// field Phi_a = sum_b J_ab s_b + h_a of every spin in phi[a]: each lane updates
// its spins a = lane, lane + 32, ... with the normalised field and its noise
// (iteration lv.sweeps of replica r), s_a <- alpha shat_a + (1 - alpha) s_a.
// Returns the sweep's largest change (every lane).
__device__ float nmfa_finish_sweep(const DevInstance& in, const DevSolve& s, int r, const Level& lv,
                                   float* m, const float* phi, int lane)
{
    float d = 0.f;
    for (int a = lane; a < in.n; a += 32) {
        const float xi = s.nmfa_sigma > 0.f
                             ? nmfa_normal(s.seed, s.stream, (uint32_t)r, (uint32_t)lv.sweeps,
                                           (uint32_t)__ldg(in.new2old + a))
                             : 0.f;
        const float v = nmfa_update(phi[a], __ldg(in.inv_norm + a), xi, s.nmfa_sigma, lv.invT,
                                    s.nmfa_alpha, m[a]);
        d = fmaxf(d, fabsf(v - m[a]));
        m[a] = v;
    }
    return warp_reduce_strided<1>(d, MaxOp());
}

__device__ __forceinline__ void init_m(const DevInstance& in, const DevSolve& s, int r, float* m,
                                       int lane)
{
    const int n = in.n;
    for (int a = lane; a < n; a += 32) {
        const int o = __ldg(in.new2old + a);
        m[a] = s.m0 ? __ldg(s.m0 + (size_t)r * n + o) : draw_m0(s.seed, s.stream, r, o);
    }
}

// Sign-round, outputs and the replica's energy (pairs a < b once plus the
// field). The lanes stride along row a, so every load of the row is
// coalesced; integer J sums exactly in int64, and for other couplings the
// library re-evaluates this sum exactly afterwards when the instance's span
// allows it.
__device__ void finish_replica(const DevInstance& in, const DevSolve& s, int r, const float* m,
                               int lane, const Level& lv)
{
    const int n = in.n;
    for (int a = lane; a < n; a += 32) {
        const int o = __ldg(in.new2old + a);
        s.sigma[(size_t)r * n + o] = (int8_t)(m[a] >= 0.f ? 1 : -1);
        if (s.m_final) s.m_final[(size_t)r * n + o] = m[a];
    }
    long long ei = 0;
    double ef = 0.0;
    for (int a = 0; a < n; ++a) {
        const int sa = m[a] >= 0.f ? 1 : -1;
        if (in.integer) {
            const int8_t* row = in.J_i8 + (size_t)a * n;
            int acc = 0;  // at most n / 32 terms of magnitude <= 128 per lane
            for (int b = a + 1 + lane; b < n; b += 32) acc += m[b] >= 0.f ? (int)row[b] : -(int)row[b];
            ei += (long long)(acc * sa);
            if (in.h && lane == 0) ei += (long long)__ldg(in.h + a) * sa;
        } else {
            const double* row = in.J_f64 + (size_t)a * n;
            double acc = 0.0;
            for (int b = a + 1 + lane; b < n; b += 32) acc += m[b] >= 0.f ? row[b] : -row[b];
            ef += acc * sa;
            if (in.h_f64 && lane == 0) ef += __ldg(in.h_f64 + a) * sa;
        }
    }
    ei = warp_reduce_strided<1>(ei, SumOp());
    ef = warp_reduce_strided<1>(ef, SumOp());
    if (lane == 0) {
        s.energy[r] = in.integer ? (double)ei : ef;
        s.energy_i64[r] = in.integer ? ei : 0;
        if (s.add_counts) {
            s.sweeps[r] += lv.sweeps;
            s.capped[r] += lv.capped;
        } else {
            s.sweeps[r] = lv.sweeps;
            s.levels[r] = lv.levels;
            s.capped[r] = lv.capped;
        }
    }
}

// The next row's cache lines are requested into L1 while this row's field is
// summed (a prefetch is a hint and never faults).
__device__ __forceinline__ void prefetch_row_l1(const float* row, int n, int lane)
{
    for (int o = lane * 32; o < n; o += 32 * 32)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(row + o));
}

// Fallback for n % 4 != 0 or n too large for the staged kernel's shared
// memory: every warp reads the rows through the read-only cache, and m lives
// in shared memory (ONCHIP) or in a global scratch row.
template <bool ONCHIP, bool JACOBI>
__global__ void __launch_bounds__(kDenseWarps * 32) dense_descent_kernel(DevInstance in, DevSolve s,
                                                                         int /*stages*/)
{
    extern __shared__ __align__(128) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * kDenseWarps + warp;
    if (r >= s.R) return;  // whole warp leaves; the kernel has no block barrier
    const int n = in.n;
    // rows (and m) start on 16-byte boundaries when n % 4 == 0: float4 path
    const int n4 = (n & 3) == 0 ? n >> 2 : 0;
    const int per = n * (JACOBI ? 2 : 1);
    float* m = ONCHIP ? smem + (size_t)warp * per : s.m_scratch + (size_t)r * per;
    float* mn = JACOBI ? m + n : m;
    init_m(in, s, r, m, lane);
    __syncwarp();
    Level lv;
    lv.start(s, r);
    while (lv.act) {
        float d = 0.f;
        for (int a = 0; a < n; ++a) {
            prefetch_row_l1(in.Jf + (size_t)(a + 1 < n ? a + 1 : 0) * n, n, lane);
            const float p = row_field<true>(in.Jf + (size_t)a * n, m, n, n4, lane,
                                            in.h && lane == 0 ? __ldg(in.h + a) : 0.f);
            // NMFA keeps the raw field; its update follows the sweep
            const float sn = JACOBI && s.nmfa ? p : -tanhf(p * lv.invT);
            if (!(JACOBI && s.nmfa)) d = fmaxf(d, fabsf(sn - m[a]));
            __syncwarp();
            if (lane == 0) mn[a] = sn;
            __syncwarp();
        }
        if (JACOBI) {
            if (s.nmfa) {
                d = nmfa_finish_sweep(in, s, r, lv, m, mn, lane);
            } else {
                for (int a = lane; a < n; a += 32) m[a] = mn[a];
            }
            __syncwarp();
        }
        lv.after_sweep(s, d);
    }
    finish_replica(in, s, r, m, lane, lv);
}

// Wait for a row stage's barrier phase. Every lane polls; the wait gives up
// when another warp has given up (abort flag) or after kSpinLimit polls, when
// it raises the flag and records the timeout in the status word.
__device__ __forceinline__ bool stage_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                           int32_t* status)
{
    for (uint32_t i = 0; i < tc::kSpinLimit; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(status, tc::kErrTimeout);
    return false;
}

// Staged kernel (n % 4 == 0): the kDenseWarps replicas of a CTA sweep the
// spins in lockstep, so each row J[a,:] is fetched once per CTA. A ring of
// `stages` row buffers in shared memory is filled by bulk copies
// (cp.async.bulk, completion on a `full` mbarrier per stage); every warp
// releases a stage on its `empty` mbarrier once its field is summed, and
// thread 0 then refills that stage with the row `stages` spins ahead. The
// rows wrap from n - 1 to 0, so the pipeline runs across sweeps; the CTA
// stops when none of its replicas is active and drains the copies still in
// flight before it exits. Warps past R take part in the pipeline only.
template <bool JACOBI>
__global__ void __launch_bounds__(kDenseWarps * 32) dense_staged_kernel(DevInstance in, DevSolve s,
                                                                        int stages)
{
    extern __shared__ __align__(128) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * kDenseWarps + warp;
    const bool live = r < s.R;
    const int n = in.n, n4 = n >> 2;
    const int per = n * (JACOBI ? 2 : 1);
    float* rows = smem;
    float* m = smem + (size_t)stages * n + (size_t)warp * per;
    float* mn = JACOBI ? m + n : m;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)stages * n + (size_t)kDenseWarps * per);
    uint64_t* empty = full + stages;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + stages);
    const uint32_t row_bytes = (uint32_t)n * sizeof(float);

    if (threadIdx.x == 0) {
        for (int k = 0; k < stages; ++k) {
            tc::mbar_init(&full[k], 1);
            tc::mbar_init(&empty[k], kDenseWarps);
        }
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < stages; ++k) {  // rows 0 .. stages - 1 (stages <= n)
            tc::mbar_arrive_expect_tx(&full[k], row_bytes);
            tc::bulk_load(rows + (size_t)k * n, in.Jf + (size_t)k * n, row_bytes, &full[k]);
        }
    Level lv;
    if (live) {
        init_m(in, s, r, m, lane);
        lv.start(s, r);
    }
    __syncwarp();

    int st = 0;        // stage of the next row to consume
    uint32_t ph = 0;   // its barrier parity
    bool any = __syncthreads_or(lv.act) != 0;
    while (any) {
        float d = 0.f;
        for (int a = 0; a < n; ++a) {
            const bool ok = __all_sync(0xffffffffu, stage_wait(&full[st], ph, abort_flag, s.status));
            if (!ok) break;
            if (lv.act) {
                const float p = row_field<false>(rows + (size_t)st * n, m, n, n4, lane,
                                                 in.h && lane == 0 ? __ldg(in.h + a) : 0.f);
                // NMFA keeps the raw field; its update follows the sweep
                const float sn = JACOBI && s.nmfa ? p : -tanhf(p * lv.invT);
                if (!(JACOBI && s.nmfa)) d = fmaxf(d, fabsf(sn - m[a]));
                __syncwarp();
                if (lane == 0) mn[a] = sn;
            }
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&empty[st]);
            if (threadIdx.x == 0 && stage_wait(&empty[st], ph, abort_flag, s.status)) {
                const int next = a + stages < n ? a + stages : a + stages - n;
                tc::mbar_arrive_expect_tx(&full[st], row_bytes);
                tc::bulk_load(rows + (size_t)st * n, in.Jf + (size_t)next * n, row_bytes, &full[st]);
            }
            if (++st == stages) {
                st = 0;
                ph ^= 1u;
            }
        }
        if (JACOBI && lv.act) {
            if (s.nmfa) {
                d = nmfa_finish_sweep(in, s, r, lv, m, mn, lane);
            } else {
                for (int a = lane; a < n; a += 32) m[a] = mn[a];
            }
            __syncwarp();
        }
        if (lv.act) lv.after_sweep(s, d);
        any = __syncthreads_or(lv.act) != 0 && !*abort_flag;
    }
    // the `stages` copies issued ahead of the last consumed row
    if (threadIdx.x == 0 && !*abort_flag)
        for (int k = 0; k < stages; ++k) {
            const int q = st + k < stages ? st + k : st + k - stages;
            if (!tc::mbar_wait(&full[q], st + k < stages ? ph : ph ^ 1u, s.status)) break;
        }
    __syncthreads();
    if (live) finish_replica(in, s, r, m, lane, lv);
}

const void* pick(const DensePlan& p, bool jacobi)
{
    if (p.stages) return jacobi ? (const void*)dense_staged_kernel<true> : (const void*)dense_staged_kernel<false>;
    if (p.onchip) return jacobi ? (const void*)dense_descent_kernel<true, true>
                                : (const void*)dense_descent_kernel<true, false>;
    return jacobi ? (const void*)dense_descent_kernel<false, true>
                  : (const void*)dense_descent_kernel<false, false>;
}

}  // namespace

DensePlan plan_dense(const DevInstance& in, int R, int jacobi, int device)
{
    int optin = 48 * 1024;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    DensePlan p;
    p.warps_per_block = kDenseWarps;
    p.grid = (R + kDenseWarps - 1) / kDenseWarps;
    const size_t per_warp = (size_t)in.n * sizeof(float) * (jacobi ? 2 : 1);
    if (in.n % 4 == 0)
        for (int stages = std::min(kMaxStages, in.n); stages >= 2 && !p.stages; --stages) {
            const size_t bytes = (size_t)stages * in.n * sizeof(float) + per_warp * kDenseWarps +
                                 2 * stages * sizeof(uint64_t) + 16;
            if (bytes <= (size_t)optin) {
                p.stages = stages;
                p.smem = bytes;
            }
        }
    if (p.stages) return p;
    p.onchip = per_warp * kDenseWarps <= (size_t)optin - 4096;
    p.smem = p.onchip ? per_warp * kDenseWarps : 0;
    p.scratch_floats = p.onchip ? 0 : (size_t)R * in.n * (jacobi ? 2 : 1);
    return p;
}

cudaError_t launch_dense(const DevInstance& in, const DevSolve& s, const DensePlan& p,
                         cudaStream_t st)
{
    const void* k = pick(p, s.jacobi != 0);
    if (p.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)p.smem);
        if (e != cudaSuccess) return e;
    }
    DevInstance a = in;
    DevSolve b = s;
    int stages = p.stages;
    void* args[] = {&a, &b, &stages};
    return cudaLaunchKernel(k, dim3(p.grid), dim3(kDenseWarps * 32), args, p.smem, st);
}

}  // namespace mars
