// Order-independent exact summation of doubles on the GPU.
//
// Energies of non-integer couplings (Section 2, Eq. 2) are sums of +-J_ij
// and +-h_i. Each term is an integer multiple of 2^e0, where e0 is the weight
// of the last mantissa bit of the smallest non-zero coupling or field, so the
// exact sum is an integer times 2^e0. The runtime picks e0 and a limb count
// per instance at ingest; a thread adds each term's 53-bit mantissa, shifted
// to its place, into base-2^32 digits held in int64 limbs (no carries until
// the end), threads combine their limbs, and one final step rounds the exact
// integer to the nearest double (ties to even). The result does not depend on
// the order of the terms.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mars {

constexpr int kExactLimbs = 8;  // 256 bits of span; enough for any Gaussian instance

struct ExactAcc {
    long long d[kExactLimbs];

    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int l = 0; l < kExactLimbs; ++l) d[l] = 0;
    }

    // Add a term whose magnitude is a multiple of 2^e0 and whose top bit lies
    // within the limbs (guaranteed by the runtime's choice of e0).
    __device__ __forceinline__ void add(double t, int e0)
    {
        if (t == 0.0) return;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(t);
        int ex = (int)((bits >> 52) & 0x7ffu);
        unsigned long long mant = bits & ((1ull << 52) - 1);
        if (ex == 0) ex = 1; else mant |= 1ull << 52;
        const int pos = ex - 1075 - e0;  // weight of mant's last bit, relative to 2^e0
        const int q = pos >> 5, r = pos & 31;
        const unsigned long long lo = mant << r;
        const unsigned long long hi = r ? (mant >> (64 - r)) : 0ull;
        long long d0 = (long long)(lo & 0xffffffffull), d1 = (long long)(lo >> 32), d2 = (long long)hi;
        if (bits >> 63) { d0 = -d0; d1 = -d1; d2 = -d2; }
#pragma unroll
        for (int l = 0; l < kExactLimbs; ++l)
            d[l] += (l == q ? d0 : 0) + (l == q + 1 ? d1 : 0) + (l == q + 2 ? d2 : 0);
    }

    // Carry-propagate so that every limb but the top one is in [0, 2^32).
    __device__ __forceinline__ void normalize()
    {
        long long carry = 0;
#pragma unroll
        for (int l = 0; l < kExactLimbs - 1; ++l) {
            const long long t = d[l] + carry;
            d[l] = t & 0xffffffffll;
            carry = (t - d[l]) >> 32;  // exact: t - low is a multiple of 2^32
        }
        d[kExactLimbs - 1] += carry;
    }

    __device__ __forceinline__ void add_acc(const ExactAcc& o)
    {
#pragma unroll
        for (int l = 0; l < kExactLimbs; ++l) d[l] += o.d[l];
    }

    // The exact value rounded to the nearest double, ties to even. The runtime
    // keeps |value| below 2^(e0 + 224), so after normalising the top limb only
    // carries the sign.
    __device__ double round(int e0)
    {
        normalize();
        const bool neg = d[kExactLimbs - 1] < 0;
        if (neg) {
#pragma unroll
            for (int l = 0; l < kExactLimbs; ++l) d[l] = -d[l];
            normalize();
        }
        int h = -1;
#pragma unroll
        for (int l = kExactLimbs - 1; l >= 0; --l)
            if (h < 0 && d[l] != 0) h = l;
        if (h < 0) return 0.0;
        auto limb = [&](int l) -> unsigned long long {
            return l >= 0 ? (unsigned long long)d[l] & 0xffffffffull : 0ull;
        };
        // W = limbs h..h-3 as a 128-bit integer; bit 0 of W weighs 2^(e0 + 32(h-3)).
        const unsigned long long whi = (limb(h) << 32) | limb(h - 1);
        const unsigned long long wlo = (limb(h - 2) << 32) | limb(h - 3);
        bool sticky = false;
        for (int l = 0; l <= h - 4; ++l) sticky |= d[l] != 0;
        // S = W << z puts the leading one at bit 127 (whi >= 2^32, so z <= 31).
        const int z = __clzll((long long)whi);
        const unsigned long long shi = z ? (whi << z) | (wlo >> (64 - z)) : whi;
        const unsigned long long slo = wlo << z;
        unsigned long long mant = shi >> 11;  // S bits 127..75
        const bool guard = (shi >> 10) & 1ull;  // S bit 74
        sticky |= (shi & 0x3ffull) != 0 || slo != 0;
        if (guard && (sticky || (mant & 1ull))) mant += 1;
        // S bit j weighs 2^(e0 + 32(h-3) + j - z); mant's last bit is S bit 75.
        const double r = ldexp((double)mant, e0 + 32 * (h - 3) + 75 - z);
        return neg ? -r : r;
    }
};

}  // namespace mars
