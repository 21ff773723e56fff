// Best-replica selection over a solve's R results, by one CTA of NT threads:
// the lowest index among the replicas of minimum energy (Section 3 keeps the
// best result of the sample), the number of replicas that reach it (the
// success count behind the paper's P, Section 4.2), the energy sum and the
// sweep, level and capped-level totals; the best replica's spins are copied.
// Used by the stand-alone argmin kernel and by the serving kernel's CTA that
// finishes a job.
#pragma once

#include "device_common.cuh"
#include "mars_internal.h"

#include <cfloat>
#include <climits>

namespace mars {

template <int NT>
__device__ void best_reduce(const DevSolve& s, int32_t n, int32_t integer, int8_t* best_spins, DevResult* res)
{
    constexpr int kW = NT / 32;
    __shared__ double s_e[kW];
    __shared__ int s_r[kW];
    __shared__ double s_sum[kW];
    __shared__ long long s_cnt[kW][4];
    __shared__ int s_best;
    __shared__ double s_beste;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double be = DBL_MAX;
    int br = INT_MAX;
    for (int r = tid; r < s.R; r += NT) {
        const double e = s.energy[r];
        if (e < be || (e == be && r < br)) { be = e; br = r; }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const double oe = __shfl_xor_sync(0xffffffffu, be, m);
        const int orr = __shfl_xor_sync(0xffffffffu, br, m);
        if (oe < be || (oe == be && orr < br)) { be = oe; br = orr; }
    }
    if (lane == 0) { s_e[warp] = be; s_r[warp] = br; }
    __syncthreads();
    if (tid == 0) {
        double e = DBL_MAX;
        int rr = INT_MAX;
        for (int w = 0; w < kW; ++w)
            if (s_e[w] < e || (s_e[w] == e && s_r[w] < rr)) { e = s_e[w]; rr = s_r[w]; }
        s_best = rr;
        s_beste = e;
    }
    __syncthreads();
    const int best = s_best;
    const double beste = s_beste;
    double sum = 0.0;
    long long hits = 0, sw = 0, lv = 0, cp = 0;
    for (int r = tid; r < s.R; r += NT) {
        const double e = s.energy[r];
        sum += e;
        hits += (e == beste);
        sw += s.sweeps[r];
        lv += s.levels[r];
        cp += s.capped[r];
    }
    sum = warp_reduce_strided<1>(sum, SumOp());
    hits = warp_reduce_strided<1>(hits, SumOp());
    sw = warp_reduce_strided<1>(sw, SumOp());
    lv = warp_reduce_strided<1>(lv, SumOp());
    cp = warp_reduce_strided<1>(cp, SumOp());
    if (lane == 0) {
        s_sum[warp] = sum;
        s_cnt[warp][0] = hits;
        s_cnt[warp][1] = sw;
        s_cnt[warp][2] = lv;
        s_cnt[warp][3] = cp;
    }
    __syncthreads();
    if (tid == 0) {
        double ts = 0.0;
        long long c[4] = {0, 0, 0, 0};
        for (int w = 0; w < kW; ++w) {
            ts += s_sum[w];
            for (int q = 0; q < 4; ++q) c[q] += s_cnt[w][q];
        }
        res->best_energy = beste;
        res->best_energy_i64 = integer ? s.energy_i64[best] : 0;
        res->best_replica = best;
        res->hits = (int32_t)c[0];
        res->sum_energy = ts;
        res->sweeps = c[1];
        res->levels = c[2];
        res->capped = c[3];
    }
    if (best_spins && best >= 0 && best < s.R)
        for (int i = tid; i < n; i += NT) best_spins[i] = s.sigma[(size_t)best * n + i];
}

}  // namespace mars
