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
