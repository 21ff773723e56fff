// Dense MARS descent (Section 3, Algorithm 1) in FP32 on the SIMT cores.
//
// One warp carries one replica through the whole descent. A sweep visits the
// spins one after another (Gauss-Seidel: every spin shares a coupling with
// every other, so there is no parallelism inside one replica's sweep); the
// warp spreads each local field Phi_a = sum_b J_ab s_b over its 32 lanes and
// reduces it with shuffles, in compensated arithmetic (see Dot2). The replica's magnetisations stay in shared memory
// when they fit, J is read through the read-only cache and shared by every
// warp on the SM. This is the plain FP32 path the tensor-core path is checked
// against; it is exact in its arithmetic order, not fast for large n.
#include "device_common.cuh"
#include "schedule.cuh"
#include "mars_internal.h"

#include <algorithm>

namespace mars {
namespace {

constexpr int kDenseWarps = 4;

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

template <bool ONCHIP, bool JACOBI>
__global__ void __launch_bounds__(kDenseWarps * 32) dense_descent_kernel(DevInstance in, DevSolve s)
{
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * kDenseWarps + warp;
    if (r >= s.R) return;  // whole warp leaves; the kernel has no block barrier
    const int n = in.n;
    const int per = n * (JACOBI ? 2 : 1);
    float* m = ONCHIP ? smem + (size_t)warp * per : s.m_scratch + (size_t)r * per;
    float* mn = JACOBI ? m + n : m;

    for (int a = lane; a < n; a += 32) {
        const int o = __ldg(in.new2old + a);
        m[a] = s.m0 ? __ldg(s.m0 + (size_t)r * n + o) : draw_m0(s.seed, s.stream, r, o);
    }
    __syncwarp();

    // the first level (schedule.cuh), or the given one (the FP32 polish)
    double T = 0.0;
    bool act;
    if (s.t_first) {
        T = s.t_first[r];
        act = T > 0.0;
    } else {
        act = sched_first(s, (double)s.t0[r], &T);
    }
    float invT = act ? sched_inv_t(T) : 0.f;
    int levels = act ? 1 : 0, sweeps = 0, capped = 0, lvl_sweeps = 0;

    while (act) {
        float d = 0.f;
        for (int a = 0; a < n; ++a) {
            const float* Jrow = in.Jf + (size_t)a * n;
            Dot2 acc;
            for (int b = lane; b < n; b += 32) acc.add_product(__ldg(Jrow + b), m[b]);
            if (in.h && lane == 0) acc.add_pair(__ldg(in.h + a), 0.f);
            const float p = acc.warp_total();
            const float sn = -tanhf(p * invT);
            d = fmaxf(d, fabsf(sn - m[a]));
            __syncwarp();
            if (lane == 0) mn[a] = sn;
            __syncwarp();
        }
        if (JACOBI) {
            for (int a = lane; a < n; a += 32) m[a] = mn[a];
            __syncwarp();
        }
        ++sweeps;
        ++lvl_sweeps;
        const bool fixed = sched_fixed(s, T);
        const bool level_done = fixed ? lvl_sweeps >= s.fixed_sweeps : (d <= s.d_min || lvl_sweeps >= s.k_max);
        if (level_done) {
            if (!fixed && !(d <= s.d_min)) ++capped;
            lvl_sweeps = 0;
            if (!s.one_level && sched_advance(s, &T)) {
                ++levels;
                invT = sched_inv_t(T);
            } else {
                act = false;
            }
        }
    }

    // sign-round, outputs and exact energy (pairs a < b once, plus the field)
    long long ei = 0;
    double ef = 0.0;
    for (int a = lane; a < n; a += 32) {
        const int sa = m[a] >= 0.f ? 1 : -1;
        const int o = __ldg(in.new2old + a);
        s.sigma[(size_t)r * n + o] = (int8_t)sa;
        if (s.m_final) s.m_final[(size_t)r * n + o] = m[a];
        if (in.integer) {
            const int8_t* row = in.J_i8 + (size_t)a * n;
            long long acc = 0;
            for (int b = a + 1; b < n; ++b) acc += (int)row[b] * (m[b] >= 0.f ? 1 : -1);
            ei += acc * sa;
            if (in.h) ei += (long long)__ldg(in.h + a) * sa;
        } else {
            const double* row = in.J_f64 + (size_t)a * n;
            double acc = 0.0;
            for (int b = a + 1; b < n; ++b) acc += row[b] * (m[b] >= 0.f ? 1.0 : -1.0);
            ef += acc * sa;
            if (in.h_f64) ef += __ldg(in.h_f64 + a) * sa;
        }
    }
    ei = warp_reduce_strided<1>(ei, SumOp());
    ef = warp_reduce_strided<1>(ef, SumOp());
    if (lane == 0) {
        s.energy[r] = in.integer ? (double)ei : ef;
        s.energy_i64[r] = in.integer ? ei : 0;
        if (s.add_counts) {
            s.sweeps[r] += sweeps;
            s.capped[r] += capped;
        } else {
            s.sweeps[r] = sweeps;
            s.levels[r] = levels;
            s.capped[r] = capped;
        }
    }
}

const void* pick(bool onchip, bool jacobi)
{
    if (onchip) return jacobi ? (const void*)dense_descent_kernel<true, true>
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
    const size_t per_warp = (size_t)in.n * sizeof(float) * (jacobi ? 2 : 1);
    p.onchip = per_warp * kDenseWarps <= (size_t)optin - 4096;
    p.smem = p.onchip ? per_warp * kDenseWarps : 0;
    p.grid = (R + kDenseWarps - 1) / kDenseWarps;
    p.scratch_floats = p.onchip ? 0 : (size_t)R * in.n * (jacobi ? 2 : 1);
    return p;
}

cudaError_t launch_dense(const DevInstance& in, const DevSolve& s, const DensePlan& p,
                         cudaStream_t st)
{
    const void* k = pick(p.onchip != 0, s.jacobi != 0);
    if (p.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)p.smem);
        if (e != cudaSuccess) return e;
    }
    DevInstance a = in;
    DevSolve b = s;
    void* args[] = {&a, &b};
    return cudaLaunchKernel(k, dim3(p.grid), dim3(kDenseWarps * 32), args, p.smem, st);
}

}  // namespace mars
