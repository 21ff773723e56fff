// Device helpers shared by the MARS kernels: the counter-based start-state
// draw and warp/block reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mars {

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
// multiplies words 0 and 2 by the two round constants, mixes the high halves
// with words 1 and 3 and the key, and the key is bumped by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t uint4_word(uint4 v, int w)
{
    return w == 0 ? v.x : w == 1 ? v.y : w == 2 ? v.z : v.w;
}

// Start magnetisation of spin `i` (caller label) in replica `r`: 2u - 1 with
// u = (word i%4 of Philox(i/4, r, 0, stream) >> 8) * 2^-24. Exact in FP32.
__device__ __forceinline__ float draw_m0(uint64_t seed, uint32_t stream, uint32_t r, uint32_t i)
{
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 out = philox4x32_10(make_uint4(i >> 2, r, 0u, stream), key);
    const float u = (float)(uint4_word(out, (int)(i & 3u)) >> 8) * 0x1p-24f;
    return __fsub_rn(__fmul_rn(2.0f, u), 1.0f);
}

// Start temperature of replica r: float(t_min + u (t_max - t_min)), u from
// word 0 of Philox(0, r, 1, stream), each double operation rounded on its own.
__device__ __forceinline__ float draw_t0(uint64_t seed, uint32_t stream, uint32_t r, double t_min,
                                         double t_max)
{
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 out = philox4x32_10(make_uint4(0u, r, 1u, stream), key);
    const double u = (double)(out.x >> 8) * 0x1p-24;
    const double prod = __dmul_rn(u, __dsub_rn(t_max, t_min));
    return __double2float_rn(__dadd_rn(t_min, prod));
}

// Noisy mean-field annealing's standard normal for replica r, iteration k and
// spin i (caller label): Philox(i/2, r, 2 + k, stream) gives words w0, w1;
// u1 = ((w0 >> 8) + 1) 2^-24 in (0, 1], u2 = (w1 >> 8) 2^-24, and the
// Box-Muller transform (Box and Muller, 1958) gives sqrt(-2 ln u1) times
// cos(2 pi u2) (even i) or sin(2 pi u2) (odd i), in FP32 with CUDA's
// accurate logf, sqrtf and sincospif.
__device__ __forceinline__ float nmfa_normal(uint64_t seed, uint32_t stream, uint32_t r, uint32_t k,
                                             uint32_t i)
{
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 w = philox4x32_10(make_uint4(i >> 1, r, 2u + k, stream), key);
    const float u1 = (float)((w.x >> 8) + 1u) * 0x1p-24f;
    const float u2 = (float)(w.y >> 8) * 0x1p-24f;
    const float rho = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    return rho * ((i & 1u) ? sn : cs);
}

// One NMFA update of a spin from its local field phi = h_i + sum_j J_ij s_j:
// alpha (-tanh((phi inv_norm + sigma xi) invT)) + (1 - alpha) s_old.
__device__ __forceinline__ float nmfa_update(float phi, float inv_norm, float xi, float sigma,
                                             float invT, float alpha, float s_old)
{
    const float shat = -tanhf(fmaf(sigma, xi, phi * inv_norm) * invT);
    return fmaf(alpha, shat - s_old, s_old);
}

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int mask)
{
    return __shfl_xor_sync(0xffffffffu, v, mask);
}

__device__ __forceinline__ long long shfl_xor(long long v, int mask)
{
    return (long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, mask);
}

// Reduce across the lanes of a warp that share (lane % stride); stride is a
// power of two <= 32. Result valid in every lane.
template <int STRIDE, typename T, typename Op>
__device__ __forceinline__ T warp_reduce_strided(T v, Op op)
{
#pragma unroll
    for (int m = 16; m >= STRIDE; m >>= 1) v = op(v, shfl_xor(v, m));
    return v;
}

struct MaxOp {
    template <typename T>
    __device__ __forceinline__ T operator()(T a, T b) const { return a > b ? a : b; }
};
struct SumOp {
    template <typename T>
    __device__ __forceinline__ T operator()(T a, T b) const { return a + b; }
};

}  // namespace mars
