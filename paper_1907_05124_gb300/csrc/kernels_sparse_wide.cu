// Sparse MARS descent (Section 3, Algorithm 1) for instances whose
// magnetisations live in global memory, level-synchronous across the grid.
//
// Every replica stays resident for the whole descent: slot q = g*RT + k of
// group g keeps its magnetisations at m[g][i*RT + k], the layout of the
// per-CTA slabs. A sweep is one launch per level of the schedule (a set of
// mutually uncoupled spins, so its updates commute and any split of the level
// over CTAs gives Algorithm 1's sequential result), then one decision launch
// that applies the stopping rule (d <= d_min or k_max sweeps) and the cooling
// step to every live replica and lists the groups still live. A level launch
// spreads (live group, 32-row slice) items over all SMs: when one replica is
// left, the whole GPU sweeps it, so a long descent no longer runs alone on
// one SM while the others idle. Each spin's field is summed in the same
// coupling order and passed through the same tanh as in the per-CTA kernels,
// so a replica's trajectory does not depend on which kernel ran it.
#include "sell_job.cuh"

#include <cstdlib>

namespace mars {
namespace {

constexpr int kWideThreads = 1024;

// Start states and per-slot schedule state. Grid-stride over
// groups x (n+1) x RT magnetisations; the first `slots` threads also set up
// their slot's level.
template <int RT>
__global__ void wide_init_kernel(DevInstance in, DevSolve s, DevWide w)
{
    const int n = in.n;
    const int64_t per_group = (int64_t)(n + 1) * RT;
    const int64_t total = per_group * w.groups;
    const int slots = w.groups * RT;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(idx / per_group);
        const int64_t rem = idx - (int64_t)g * per_group;
        const int i = (int)(rem / RT), k = (int)(rem % RT);
        const int r = s.tile_rep[g * RT + k];
        float v = 0.f;
        if (i < n && r >= 0) {
            const int o = __ldg(in.new2old + i);
            v = s.m0 ? __ldg(s.m0 + (size_t)r * n + o) : draw_m0(s.seed, s.stream, r, o);
        }
        w.m[(size_t)g * w.slab + rem] = v;
        if (idx < slots) {
            const int q = (int)idx;
            const int rq = s.tile_rep[q];
            double T = 0.0;
            const bool act = rq >= 0 && sched_first(s, (double)s.t0[rq], &T);
            w.T[q] = T;
            w.invT[q] = act ? sched_inv_t(T) : 0.f;
            w.live[q] = act;
            w.levels[q] = act ? 1 : 0;
            w.lvl_sweeps[q] = 0;
            w.sweeps[q] = 0;
            w.capped[q] = 0;
            w.dmax[q] = 0u;
        }
    }
}

// The largest |change| of a warp's items for each slot of group g, folded
// into the slot's sweep maximum (non-negative floats order like their bits).
template <int RT>
__device__ __forceinline__ void flush_d(const DevWide& w, int g, int live, float (&dloc)[RT], int lane)
{
#pragma unroll
    for (int k = 0; k < RT; ++k) {
        const float v = warp_reduce_strided<1>(dloc[k], MaxOp());
        if (lane == 0 && ((live >> k) & 1) && v > 0.f) atomicMax(w.dmax + g * RT + k, __float_as_uint(v));
        dloc[k] = 0.f;
    }
}

// One level of one sweep for every live replica. The items (live group,
// slice of the level) are cut into one contiguous chunk per CTA, and the
// CTA's warps take the chunk's items in turn. A lane owns one row of a slice
// and updates it for the group's RT slots from one walk over its couplings:
// the RT-wide gathers of the neighbours' magnetisations serve every slot.
template <int RT, int FMT, int DEG>
__global__ void __launch_bounds__(kWideThreads, 1) wide_level_kernel(DevInstance in, DevSolve s, DevWide w,
                                                                        int l)
{
    (void)s;
    using V = Vec<RT>;
    constexpr int kWarps = kWideThreads / 32;
    const int ng = w.counters[0];
    if (ng == 0) return;
    const int s0 = __ldg(in.lvl_slice + l), s1 = __ldg(in.lvl_slice + l + 1);
    const int nsl = s1 - s0;
    if (nsl <= 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Entry<FMT> ent;
    if constexpr (FMT == 0) ent.e = in.sell_gen;
    if constexpr (FMT == 1) ent.e = in.sell_pm1;
    const int64_t items = (int64_t)ng * nsl;
    const int64_t per = (items + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per;
    const int64_t b1 = b0 + per < items ? b0 + per : items;

    int cur = -1, live = 0;
    bool lean = false;
    float invT[RT], dloc[RT];
    float* m = nullptr;
#pragma unroll
    for (int k = 0; k < RT; ++k) { invT[k] = 0.f; dloc[k] = 0.f; }
    if constexpr (FMT == 1 && DEG > 0) {
        // Every row has degree DEG, so every slice does: slice sl of the level
        // starts at row dA.x + 32 (sl - s0) and its couplings at
        // dA.w + 32 DEG (sl - s0). With no descriptor to wait for, the next
        // item's coupling words and group are loaded while this item's
        // neighbour gathers are in flight, leaving one round trip per item.
        const int4 dA = __ldg(in.slices + s0);
        const int4 dB = __ldg(in.slices + s1 - 1);
        const int row_end = dB.x + dB.y;
        const uint32_t* ew = in.sell_pm1 + dA.w + lane;
        int64_t it = b0 + warp;
        uint32_t cw[DEG];
        int g = 0, sl = 0;
        if (it < b1) {
            const int gi = (int)(it / nsl);
            sl = (int)(it - (int64_t)gi * nsl);
            g = __ldg(w.glist + gi);
#pragma unroll
            for (int q = 0; q < DEG; ++q) cw[q] = __ldg(ew + (size_t)sl * 32 * DEG + 32 * q);
        }
        while (it < b1) {
            const int64_t itn = it + kWarps;
            uint32_t cn[DEG];
            int gn = g, sln = 0;
            if (itn < b1) {
                const int gi = (int)(itn / nsl);
                sln = (int)(itn - (int64_t)gi * nsl);
                gn = __ldg(w.glist + gi);
#pragma unroll
                for (int q = 0; q < DEG; ++q) cn[q] = __ldg(ew + (size_t)sln * 32 * DEG + 32 * q);
            } else {
#pragma unroll
                for (int q = 0; q < DEG; ++q) cn[q] = 0u;
            }
            if (g != cur) {
                if (cur >= 0) flush_d<RT>(w, cur, live, dloc, lane);
                cur = g;
                m = w.m + (size_t)g * w.slab;
                live = 0;
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    invT[k] = w.invT[g * RT + k];
                    live |= w.live[g * RT + k] ? 1 << k : 0;
                }
                lean = live == (1 << RT) - 1 && !in.h;
            }
            const int i = dA.x + 32 * sl + lane;
            if (i < row_end) {
                const typename V::T old = V::load(m + i * RT);
                const float hv = in.h ? __ldg(in.h + i) : 0.f;
                typename V::T acc;
#pragma unroll
                for (int k = 0; k < RT; ++k) V::set(acc, k, 0.f);
#pragma unroll
                for (int q = 0; q < DEG; ++q) {
                    const int c = (int)(cw[q] & 0x7fffffffu);
                    const float wt = (cw[q] >> 31) ? -1.f : 1.f;
                    const typename V::T mv = V::load(m + c * RT);
#pragma unroll
                    for (int k = 0; k < RT; ++k) V::set(acc, k, fmaf(wt, V::get(mv, k), V::get(acc, k)));
                }
                typename V::T nv;
                if (lean) {
#pragma unroll
                    for (int k = 0; k < RT; ++k) {
                        const float sn = -tanh_sfu(V::get(acc, k) * invT[k]);
                        dloc[k] = fmaxf(dloc[k], fabsf(sn - V::get(old, k)));
                        V::set(nv, k, sn);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < RT; ++k) {
                        if ((live >> k) & 1) {
                            const float sn = -tanh_sfu((V::get(acc, k) + hv) * invT[k]);
                            dloc[k] = fmaxf(dloc[k], fabsf(sn - V::get(old, k)));
                            V::set(nv, k, sn);
                        } else {
                            V::set(nv, k, V::get(old, k));
                        }
                    }
                }
                V::store(m + i * RT, nv);
            }
            it = itn;
            g = gn;
            sl = sln;
#pragma unroll
            for (int q = 0; q < DEG; ++q) cw[q] = cn[q];
        }
        if (cur >= 0) flush_d<RT>(w, cur, live, dloc, lane);
        return;
    } else {
    for (int64_t it = b0 + warp; it < b1; it += kWarps) {
        const int gi = (int)(it / nsl);
        const int sl = s0 + (int)(it - (int64_t)gi * nsl);
        const int g = __ldg(w.glist + gi);
        if (g != cur) {
            if (cur >= 0) flush_d<RT>(w, cur, live, dloc, lane);
            cur = g;
            m = w.m + (size_t)g * w.slab;
            live = 0;
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                invT[k] = w.invT[g * RT + k];
                live |= w.live[g * RT + k] ? 1 << k : 0;
            }
            lean = live == (1 << RT) - 1 && !in.h;
        }
        const int4 d = __ldg(in.slices + sl);  // row0, rows, degree, offset
        if (lane < d.y) {
            const int i = d.x + lane;
            const float hv = in.h ? __ldg(in.h + i) : 0.f;
            typename V::T acc;
#pragma unroll
            for (int k = 0; k < RT; ++k) V::set(acc, k, 0.f);
            const int deg = DEG > 0 ? DEG : d.z;
#pragma unroll 4
            for (int q = 0; q < deg; ++q) {
                int c;
                float wt;
                ent.get(d.w + 32 * q + lane, c, wt);
                const typename V::T mv = V::load(m + c * RT);
#pragma unroll
                for (int k = 0; k < RT; ++k) V::set(acc, k, fmaf(wt, V::get(mv, k), V::get(acc, k)));
            }
            const typename V::T old = V::load(m + i * RT);
            typename V::T nv;
            if (lean) {
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    const float sn = -tanh_sfu(V::get(acc, k) * invT[k]);
                    dloc[k] = fmaxf(dloc[k], fabsf(sn - V::get(old, k)));
                    V::set(nv, k, sn);
                }
            } else {
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    if ((live >> k) & 1) {
                        const float sn = -tanh_sfu((V::get(acc, k) + hv) * invT[k]);
                        dloc[k] = fmaxf(dloc[k], fabsf(sn - V::get(old, k)));
                        V::set(nv, k, sn);
                    } else {
                        V::set(nv, k, V::get(old, k));
                    }
                }
            }
            V::store(m + i * RT, nv);
        }
    }
    if (cur >= 0) flush_d<RT>(w, cur, live, dloc, lane);
    }
}

// Shared memory of the staged level kernel: two stages per warp, each holding
// one item's DEG x 32 RT-wide neighbour gathers.
template <int RT, int DEG>
constexpr size_t staged_smem_bytes()
{
    return (size_t)(kWideThreads / 32) * 2 * DEG * 32 * RT * sizeof(float);
}

template <int BYTES>
__device__ __forceinline__ void cp_async_ca(uint32_t dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The level kernel for regular +-1 lattices with the neighbour gathers staged
// in shared memory: while a warp computes item j from its stage, the
// asynchronous copies of item j+1's gathers (which hold no registers) and the
// coupling words of item j+2 are in flight, so each SM keeps about twice the
// loads of the register-pipelined kernel outstanding. The arithmetic per spin
// is the same: the couplings in order, the same tanh.
template <int RT, int DEG>
__global__ void __launch_bounds__(kWideThreads, 1) wide_level_staged_kernel(DevInstance in, DevSolve s,
                                                                               DevWide w, int l)
{
    (void)s;
    using V = Vec<RT>;
    constexpr int kWarps = kWideThreads / 32;
    constexpr int kStage = DEG * 32 * RT;  // floats of one stage
    extern __shared__ float4 wide_stage_smem[];
    const int ng = w.counters[0];
    if (ng == 0) return;
    const int s0 = __ldg(in.lvl_slice + l), s1 = __ldg(in.lvl_slice + l + 1);
    const int nsl = s1 - s0;
    if (nsl <= 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t items = (int64_t)ng * nsl;
    const int64_t per = (items + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * per;
    const int64_t b1 = b0 + per < items ? b0 + per : items;
    int64_t itA = b0 + warp;
    if (itA >= b1) return;  // no barrier follows: a warp without items may leave

    // Slice sl of the level: rows dA.x + 32 sl .., couplings at dA.w + 32 DEG sl.
    const int4 dA = __ldg(in.slices + s0);
    const int4 dB = __ldg(in.slices + s1 - 1);
    const int row_end = dB.x + dB.y;
    const uint32_t* ew = in.sell_pm1 + dA.w + lane;
    float* const stage0 = reinterpret_cast<float*>(wide_stage_smem) + (size_t)warp * 2 * kStage;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(stage0);

    // Copies item (g, sl)'s gathers into stage st; returns the sign bits.
    uint32_t cw[DEG];
    auto issue = [&](int g, int st) -> uint32_t {
        const float* mg = w.m + (size_t)g * w.slab;
        uint32_t signs = 0;
#pragma unroll
        for (int q = 0; q < DEG; ++q) {
            const int c = (int)(cw[q] & 0x7fffffffu);
            signs |= (cw[q] >> 31) << q;
            cp_async_ca<RT * 4>(sbase + (uint32_t)((st * kStage + (q * 32 + lane) * RT) * sizeof(float)),
                                mg + (size_t)c * RT);
        }
        return signs;
    };
    auto couplings = [&](int sl) {
#pragma unroll
        for (int q = 0; q < DEG; ++q) cw[q] = __ldg(ew + (size_t)sl * 32 * DEG + 32 * q);
    };
    auto old_of = [&](int g, int sl) {
        typename V::T v;
        const int i = dA.x + 32 * sl + lane;
        if (i < row_end) {
            v = V::load(w.m + (size_t)g * w.slab + (size_t)i * RT);
        } else {
#pragma unroll
            for (int k = 0; k < RT; ++k) V::set(v, k, 0.f);
        }
        return v;
    };

    int gA = 0, slA = 0;
    {
        const int gi = (int)(itA / nsl);
        slA = (int)(itA - (int64_t)gi * nsl);
        gA = __ldg(w.glist + gi);
    }
    couplings(slA);
    uint32_t signA = issue(gA, 0);
    cp_async_commit();
    typename V::T oldA = old_of(gA, slA);
    int64_t itB = itA + kWarps;
    bool hasB = itB < b1;
    int gB = gA, slB = 0;
    if (hasB) {
        const int gi = (int)(itB / nsl);
        slB = (int)(itB - (int64_t)gi * nsl);
        gB = __ldg(w.glist + gi);
        couplings(slB);
    }

    int cur = -1, live = 0, st = 0;
    bool lean = false;
    float invT[RT], dloc[RT];
    float* m = nullptr;
#pragma unroll
    for (int k = 0; k < RT; ++k) { invT[k] = 0.f; dloc[k] = 0.f; }
    for (;;) {
        uint32_t signB = 0;
        typename V::T oldB;
        if (hasB) {
            signB = issue(gB, st ^ 1);
            oldB = old_of(gB, slB);
        }
        cp_async_commit();
        const int64_t itC = itB + kWarps;
        const bool hasC = hasB && itC < b1;
        int gC = gB, slC = 0;
        if (hasC) {
            const int gi = (int)(itC / nsl);
            slC = (int)(itC - (int64_t)gi * nsl);
            gC = __ldg(w.glist + gi);
            couplings(slC);
        }
        cp_async_wait<1>();  // item A's copies have landed
        if (gA != cur) {
            if (cur >= 0) flush_d<RT>(w, cur, live, dloc, lane);
            cur = gA;
            m = w.m + (size_t)gA * w.slab;
            live = 0;
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                invT[k] = w.invT[gA * RT + k];
                live |= w.live[gA * RT + k] ? 1 << k : 0;
            }
            lean = live == (1 << RT) - 1 && !in.h;
        }
        const int i = dA.x + 32 * slA + lane;
        if (i < row_end) {
            const float* sg = stage0 + st * kStage + lane * RT;
            const float hv = in.h ? __ldg(in.h + i) : 0.f;
            typename V::T acc;
#pragma unroll
            for (int k = 0; k < RT; ++k) V::set(acc, k, 0.f);
#pragma unroll
            for (int q = 0; q < DEG; ++q) {
                const float wt = ((signA >> q) & 1u) ? -1.f : 1.f;
                const typename V::T mv = V::load(sg + q * 32 * RT);
#pragma unroll
                for (int k = 0; k < RT; ++k) V::set(acc, k, fmaf(wt, V::get(mv, k), V::get(acc, k)));
            }
            typename V::T nv;
            if (lean) {
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    const float sn = -tanh_sfu(V::get(acc, k) * invT[k]);
                    dloc[k] = fmaxf(dloc[k], fabsf(sn - V::get(oldA, k)));
                    V::set(nv, k, sn);
                }
            } else {
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    if ((live >> k) & 1) {
                        const float sn = -tanh_sfu((V::get(acc, k) + hv) * invT[k]);
                        dloc[k] = fmaxf(dloc[k], fabsf(sn - V::get(oldA, k)));
                        V::set(nv, k, sn);
                    } else {
                        V::set(nv, k, V::get(oldA, k));
                    }
                }
            }
            V::store(m + (size_t)i * RT, nv);
        }
        if (!hasB) break;
        gA = gB;
        slA = slB;
        signA = signB;
        oldA = oldB;
        gB = gC;
        slB = slC;
        hasB = hasC;
        itB = itC;
        st ^= 1;
    }
    cp_async_wait<0>();
    if (cur >= 0) flush_d<RT>(w, cur, live, dloc, lane);
}

// After a sweep (step != 0): each live slot's sweep count, the stopping rule
// on its largest change d, and the cooling step, as in the per-CTA kernels;
// then (also with step == 0, after the start) the live groups in ascending
// order and the live group and replica counts. One CTA.
__global__ void __launch_bounds__(kWideThreads) wide_decide_kernel(DevSolve s, DevWide w, int step)
{
    __shared__ int s_cnt[kWideThreads];
    __shared__ int s_warp[kWideThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int slots = w.groups * w.rt;
    if (step) {
        for (int q = tid; q < slots; q += kWideThreads) {
            if (!w.live[q]) continue;
            const float dd = __uint_as_float(w.dmax[q]);
            w.dmax[q] = 0u;
            int ls = w.lvl_sweeps[q] + 1;
            w.sweeps[q] += 1;
            double T = w.T[q];
            const bool fixed = sched_fixed(s, T);
            const bool level_done = fixed ? ls >= s.fixed_sweeps : (dd <= s.d_min || ls >= s.k_max);
            if (level_done) {
                if (!fixed && !(dd <= s.d_min)) w.capped[q] += 1;
                ls = 0;
                if (sched_advance(s, &T)) {
                    w.T[q] = T;
                    w.levels[q] += 1;
                    w.invT[q] = sched_inv_t(T);
                } else {
                    w.live[q] = 0;
                }
            }
            w.lvl_sweeps[q] = ls;
        }
        __syncthreads();
    }
    // ordered compaction: thread t owns the groups [t*per, (t+1)*per)
    const int G = w.groups;
    const int per = (G + kWideThreads - 1) / kWideThreads;
    const int g0 = tid * per, g1 = min(G, g0 + per);
    int cnt = 0, reps = 0;
    for (int g = g0; g < g1; ++g) {
        int any = 0;
        for (int k = 0; k < w.rt; ++k) any += w.live[g * w.rt + k] != 0;
        reps += any;
        cnt += any > 0;
    }
    // exclusive scan of cnt over the block
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    s_cnt[tid] = reps;
    __syncthreads();
    if (warp == 0) {
        int v = lane < kWideThreads / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < kWideThreads / 32) s_warp[lane] = v;  // inclusive warp totals
    }
    __syncthreads();
    int pos = x - cnt + (warp > 0 ? s_warp[warp - 1] : 0);
    for (int g = g0; g < g1; ++g) {
        int any = 0;
        for (int k = 0; k < w.rt; ++k) any |= w.live[g * w.rt + k];
        if (any) w.glist[pos++] = g;
    }
    // live replicas: a plain block sum
    for (int o = kWideThreads / 2; o > 0; o >>= 1) {
        __syncthreads();
        if (tid < o) s_cnt[tid] += s_cnt[tid + o];
    }
    if (tid == 0) {
        w.counters[0] = s_warp[kWideThreads / 32 - 1];
        w.counters[1] = s_cnt[0];
    }
}

// Outputs of every replica once the descent is over: sign-rounded spins and
// final magnetisations in caller labels, the energy of the spins (exact for
// integer couplings; FP64 sums otherwise, summed in the per-CTA kernels'
// order), and the replica's sweep, level and capped-level counts. One CTA per
// slot at a time.
template <int RT>
__global__ void __launch_bounds__(kWideThreads) wide_finalize_kernel(DevInstance in, DevSolve s, DevWide w)
{
    __shared__ long long s_ei[kWideThreads / 32];
    __shared__ double s_ef[kWideThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = in.n;
    const int slots = w.groups * RT;
    for (int q = blockIdx.x; q < slots; q += gridDim.x) {
        const int r = s.tile_rep[q];
        if (r < 0) continue;
        const int k = q % RT;
        const float* m = w.m + (size_t)(q / RT) * w.slab;
        long long ei = 0;
        double ef = 0.0;
        for (int i = tid; i < n; i += kWideThreads) {
            const int o = __ldg(in.new2old + i);
            const float mv = m[i * RT + k];
            s.sigma[(size_t)r * n + o] = (int8_t)(mv >= 0.f ? 1 : -1);
            if (s.m_final) s.m_final[(size_t)r * n + o] = mv;
            const bool pi = mv >= 0.f;
            const int e0 = __ldg(in.row_ptr + i), e1 = __ldg(in.row_ptr + i + 1);
            for (int e = e0; e < e1; ++e) {
                const int j = __ldg(in.col + e);
                if (j <= i) continue;
                const bool pj = m[j * RT + k] >= 0.f;
                if (in.integer) {
                    const int wt = (int)__ldg(in.val_i8 + e);
                    ei += pi == pj ? wt : -wt;
                } else {
                    const double wt = __ldg(in.val_f64 + e);
                    ef += pi == pj ? wt : -wt;
                }
            }
            const int si = pi ? 1 : -1;
            if (in.integer) {
                if (in.h) ei += (long long)__ldg(in.h + i) * si;
            } else if (in.h_f64) {
                ef += __ldg(in.h_f64 + i) * si;
            }
        }
        const long long a = warp_reduce_strided<1>(ei, SumOp());
        const double b = warp_reduce_strided<1>(ef, SumOp());
        if (lane == 0) { s_ei[warp] = a; s_ef[warp] = b; }
        __syncthreads();
        if (tid == 0) {
            long long ti = 0;
            double tf = 0.0;
            for (int v = 0; v < kWideThreads / 32; ++v) { ti += s_ei[v]; tf += s_ef[v]; }
            s.energy[r] = in.integer ? (double)ti : tf;
            s.energy_i64[r] = in.integer ? ti : 0;
            s.sweeps[r] = w.sweeps[q];
            s.levels[r] = w.levels[q];
            s.capped[r] = w.capped[q];
        }
        __syncthreads();
    }
}

template <int RT>
const void* pick_level_rt(int fmt, int deg)
{
    if (fmt == 0) return (const void*)wide_level_kernel<RT, 0, 0>;
    return deg == 4 ? (const void*)wide_level_kernel<RT, 1, 4>
         : deg == 6 ? (const void*)wide_level_kernel<RT, 1, 6>
                    : (const void*)wide_level_kernel<RT, 1, 0>;
}

const void* pick_level(int rt, int fmt, int deg)
{
    switch (rt) {
    case 1: return pick_level_rt<1>(fmt, deg);
    case 2: return pick_level_rt<2>(fmt, deg);
    case 4: return pick_level_rt<4>(fmt, deg);
    }
    return nullptr;
}

// The staged kernel (regular +-1 lattices) and its shared memory, or null.
template <int RT>
const void* pick_staged_rt(int deg, size_t* smem)
{
    if (deg == 4) { *smem = staged_smem_bytes<RT, 4>(); return (const void*)wide_level_staged_kernel<RT, 4>; }
    if (deg == 6) { *smem = staged_smem_bytes<RT, 6>(); return (const void*)wide_level_staged_kernel<RT, 6>; }
    return nullptr;
}

const void* pick_staged(int rt, int fmt, int deg, size_t* smem)
{
    *smem = 0;
    if (fmt != 1) return nullptr;
    switch (rt) {
    case 1: return pick_staged_rt<1>(deg, smem);
    case 2: return pick_staged_rt<2>(deg, smem);
    case 4: return pick_staged_rt<4>(deg, smem);
    }
    return nullptr;
}

const void* pick_init(int rt)
{
    return rt == 1 ? (const void*)wide_init_kernel<1> : rt == 2 ? (const void*)wide_init_kernel<2>
                                                                : (const void*)wide_init_kernel<4>;
}

const void* pick_finalize(int rt)
{
    return rt == 1 ? (const void*)wide_finalize_kernel<1> : rt == 2 ? (const void*)wide_finalize_kernel<2>
                                                                    : (const void*)wide_finalize_kernel<4>;
}

}  // namespace

bool plan_sparse_wide(const DevInstance& in, int R, int rt, int device, WidePlan* p)
{
    if (!in.slices || (!in.sell_pm1 && !in.sell_gen)) return false;
    if (rt != 1 && rt != 2 && rt != 4) return false;
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    p->rt = rt;
    p->entry = in.sell_pm1 ? 1 : 0;
    p->deg = p->entry == 1 ? in.regular_deg : 0;
    if (p->deg != 4 && p->deg != 6) p->deg = 0;
    p->groups = (R + rt - 1) / rt;
    p->slab = sell_slab_floats(in.n, rt);
    const void* k = pick_level(rt, p->entry, p->deg);
    p->smem = 0;
    p->staged = 0;
    if (const char* e = std::getenv("MARS_WIDE_STAGED"); !e || std::atoi(e) != 0) {
        size_t sm = 0;
        if (const void* ks = pick_staged(rt, p->entry, p->deg, &sm)) {
            if (cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) == cudaSuccess) {
                k = ks;
                p->smem = sm;
                p->staged = 1;
            }
        }
    }
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kWideThreads, p->smem);
    p->grid = sms * (per_sm > 0 ? per_sm : 1);
    p->sms = sms;
    return true;
}

cudaError_t launch_wide_init(const DevInstance& in, const DevSolve& s, const DevWide& w, const WidePlan& p,
                             cudaStream_t st)
{
    DevInstance a = in;
    DevSolve b = s;
    DevWide c = w;
    void* args[] = {&a, &b, &c};
    return cudaLaunchKernel(pick_init(p.rt), dim3(p.sms * 4), dim3(256), args, 0, st);
}

cudaError_t launch_wide_level(const DevInstance& in, const DevSolve& s, const DevWide& w, const WidePlan& p,
                              int level, cudaStream_t st)
{
    DevInstance a = in;
    DevSolve b = s;
    DevWide c = w;
    int l = level;
    void* args[] = {&a, &b, &c, &l};
    size_t sm = 0;
    const void* k = p.staged ? pick_staged(p.rt, p.entry, p.deg, &sm) : pick_level(p.rt, p.entry, p.deg);
    if (!k) return cudaErrorInvalidValue;
    return cudaLaunchKernel(k, dim3(p.grid), dim3(kWideThreads), args, p.smem, st);
}

cudaError_t launch_wide_decide(const DevSolve& s, const DevWide& w, int step, cudaStream_t st)
{
    DevSolve b = s;
    DevWide c = w;
    int k = step;
    void* args[] = {&b, &c, &k};
    return cudaLaunchKernel((const void*)wide_decide_kernel, dim3(1), dim3(kWideThreads), args, 0, st);
}

cudaError_t launch_wide_finalize(const DevInstance& in, const DevSolve& s, const DevWide& w, const WidePlan& p,
                                 cudaStream_t st)
{
    DevInstance a = in;
    DevSolve b = s;
    DevWide c = w;
    void* args[] = {&a, &b, &c};
    const int slots = w.groups * p.rt;
    const int grid = slots < p.sms * 2 ? slots : p.sms * 2;
    return cudaLaunchKernel(pick_finalize(p.rt), dim3(grid > 0 ? grid : 1), dim3(kWideThreads), args, 0, st);
}

}  // namespace mars
