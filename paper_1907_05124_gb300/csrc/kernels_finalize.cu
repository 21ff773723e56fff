// Start-state draw, best-replica selection and energies of given spins.
//
// The best replica is the lowest index among the replicas of minimum energy
// (Section 3: the best result of the sample is kept); hits counts the
// replicas that reach it, as the paper's success probability P does
// (Section 4.2). Energies are Eq. 2 with each pair counted once.
#include "device_common.cuh"
#include "best_reduce.cuh"
#include "exact_sum.cuh"
#include "mars_internal.h"

#include <cfloat>
#include <climits>

namespace mars {
namespace {

__global__ void draw_kernel(uint64_t seed, uint32_t stream, int32_t r0, int32_t R, int32_t n,
                            double t_min, double t_max, float* m0, float* t0)
{
    const size_t total = (size_t)R * n;
    const size_t step = (size_t)gridDim.x * blockDim.x;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += step) {
        const uint32_t q = (uint32_t)(idx / n), i = (uint32_t)(idx % n);
        if (m0) m0[idx] = draw_m0(seed, stream, (uint32_t)r0 + q, i);
    }
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < (size_t)R; q += step)
        if (t0) t0[q] = draw_t0(seed, stream, (uint32_t)(r0 + q), t_min, t_max);
}

constexpr int kBestThreads = 1024;

__global__ void __launch_bounds__(kBestThreads) best_kernel(DevSolve s, int32_t n, int32_t integer,
                                                            int8_t* best_spins, DevResult* res)
{
    best_reduce<kBestThreads>(s, n, integer, best_spins, res);
}

constexpr int kEnergyThreads = 256;

// Energies of spin vectors, one CTA per vector. Integer couplings sum exactly
// in int64; other couplings sum exactly in an ExactAcc and are rounded once.
__global__ void __launch_bounds__(kEnergyThreads) energy_kernel(DevInstance in, const int8_t* spins,
                                                                double* e, long long* e_i64,
                                                                int32_t* status)
{
    __shared__ long long s_i[kEnergyThreads / 32];
    __shared__ double s_f[kEnergyThreads / 32];
    __shared__ long long s_x[kEnergyThreads / 32][kExactLimbs];
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = in.n;
    const int8_t* sp = spins + (size_t)c * n;
    long long ei = 0;
    double ef = 0.0;  // plain FP64 sum when the instance's span exceeds the accumulator
    const bool exact = in.exact_ok != 0;
    ExactAcc ex;
    ex.clear();
    for (int a = tid; a < n; a += kEnergyThreads) {
        const int sa = sp[__ldg(in.new2old + a)];
        if (sa != 1 && sa != -1) { atomicExch(status, (int)kDevBadIndex); continue; }
        if (in.dense) {
            if (in.integer) {
                const int8_t* row = in.J_i8 + (size_t)a * n;
                long long acc = 0;
                for (int b = a + 1; b < n; ++b) acc += (int)row[b] * (int)sp[__ldg(in.new2old + b)];
                ei += acc * sa;
            } else {
                const double* row = in.J_f64 + (size_t)a * n;
                for (int b = a + 1; b < n; ++b) {
                    const double w = sa * sp[__ldg(in.new2old + b)] > 0 ? row[b] : -row[b];
                    if (exact) ex.add(w, in.exact_e0); else ef += w;
                }
            }
        } else {
            const int e0 = __ldg(in.row_ptr + a), e1 = __ldg(in.row_ptr + a + 1);
            if (in.integer) {
                long long acc = 0;
                for (int q = e0; q < e1; ++q) {
                    const int b = __ldg(in.col + q);
                    if (b > a) acc += (int)__ldg(in.val_i8 + q) * (int)sp[__ldg(in.new2old + b)];
                }
                ei += acc * sa;
            } else {
                for (int q = e0; q < e1; ++q) {
                    const int b = __ldg(in.col + q);
                    if (b <= a) continue;
                    const double v = __ldg(in.val_f64 + q);
                    const double w = sa * sp[__ldg(in.new2old + b)] > 0 ? v : -v;
                    if (exact) ex.add(w, in.exact_e0); else ef += w;
                }
            }
        }
        if (in.integer) {
            if (in.h) ei += (long long)__ldg(in.h + a) * sa;
        } else if (in.h_f64) {
            const double hv = sa > 0 ? __ldg(in.h_f64 + a) : -__ldg(in.h_f64 + a);
            if (exact) ex.add(hv, in.exact_e0); else ef += hv;
        }
    }
    ei = warp_reduce_strided<1>(ei, SumOp());
    ef = warp_reduce_strided<1>(ef, SumOp());
    ex.normalize();  // limbs small enough that 256 of them sum without overflow
#pragma unroll
    for (int l = 0; l < kExactLimbs; ++l) ex.d[l] = warp_reduce_strided<1>(ex.d[l], SumOp());
    if (lane == 0) {
        s_i[warp] = ei;
        s_f[warp] = ef;
#pragma unroll
        for (int l = 0; l < kExactLimbs; ++l) s_x[warp][l] = ex.d[l];
    }
    __syncthreads();
    if (tid == 0) {
        long long ti = 0;
        double tf = 0.0;
        ExactAcc tot;
        tot.clear();
        for (int w = 0; w < kEnergyThreads / 32; ++w) {
            ti += s_i[w];
            tf += s_f[w];
#pragma unroll
            for (int l = 0; l < kExactLimbs; ++l) tot.d[l] += s_x[w][l];
        }
        e[c] = in.integer ? (double)ti : exact ? tot.round(in.exact_e0) : tf;
        if (e_i64) e_i64[c] = in.integer ? ti : 0;
    }
}

// Replica queue in index order (entries past R empty), counters at zero.
__global__ void queue_identity_kernel(int32_t* q, int32_t total, int32_t R, int32_t* counters)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x)
        q[i] = i < R ? i : -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        counters[0] = 0;
        counters[1] = 0;
    }
}

}  // namespace

cudaError_t launch_queue_identity(int32_t* q, int32_t total, int32_t R, int32_t* counters,
                                  cudaStream_t st)
{
    queue_identity_kernel<<<(total + 255) / 256, 256, 0, st>>>(q, total, R, counters);
    return cudaGetLastError();
}

cudaError_t launch_draw(uint64_t seed, uint32_t stream, int32_t r0, int32_t R, int32_t n,
                        double t_min, double t_max, float* m0, float* t0, cudaStream_t st)
{
    const size_t total = (size_t)R * (n > 0 ? n : 1);
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    draw_kernel<<<blocks, 256, 0, st>>>(seed, stream, r0, R, n, t_min, t_max, m0, t0);
    return cudaGetLastError();
}

cudaError_t launch_best(const DevSolve& s, int32_t n, int32_t integer, int8_t* best_spins,
                        DevResult* res, cudaStream_t st)
{
    best_kernel<<<1, kBestThreads, 0, st>>>(s, n, integer, best_spins, res);
    return cudaGetLastError();
}

cudaError_t launch_energy(const DevInstance& in, const int8_t* spins, int32_t count, double* e,
                          long long* e_i64, int32_t* status, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    energy_kernel<<<count, kEnergyThreads, 0, st>>>(in, spins, e, e_i64, status);
    return cudaGetLastError();
}

// Failure detection's bounded wait (mars_device_check): poll a flag in
// host-mapped memory with a clock64 budget. Nothing is in flight while it
// waits, so giving up is only a status word and a return.
__global__ void flag_wait_kernel(const volatile int32_t* flag, long long budget_cycles, int32_t* status)
{
    const long long t0 = clock64();
    int32_t seen = 0;
    while (!(seen = *flag) && clock64() - t0 < budget_cycles) __nanosleep(200);
    *status = seen ? kDevOk : kDevTimeout;
}

cudaError_t launch_flag_wait(const int32_t* flag, long long budget_cycles, int32_t* status,
                             cudaStream_t st)
{
    flag_wait_kernel<<<1, 1, 0, st>>>(flag, budget_cycles, status);
    return cudaGetLastError();
}

}  // namespace mars
