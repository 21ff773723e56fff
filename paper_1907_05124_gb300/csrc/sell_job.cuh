// One sliced-ELL descent job (Section 3, Algorithm 1), shared by the sparse
// kernels: the coupling formats, the RT-wide replica vectors, the per-CTA
// slot bookkeeping and run_job, which drains one instance's replica queue on
// a CTA. The kernels differ only in where the magnetisations m[i*RT + k]
// live: shared memory (kernels_sparse_sell.cu) or a slab of global memory
// per CTA (kernels_sparse_slab.cu); run_job addresses them through a plain
// pointer either way.
#pragma once

#include "best_reduce.cuh"
#include "device_common.cuh"
#include "schedule.cuh"
#include "mars_internal.h"

namespace mars {
namespace {


// tanh(x) = sign(x) (1 - 2 / (1 + e^{2|x|})), with e^{2|x|} = 2^{2|x| log2 e}
// from the SFU's ex2.approx and the quotient from its rcp.approx. Absolute
// error below 2.5e-7 over all of R (checked against FP64 tanh through the C
// ABI by the fields-only test); saturates to +-1 when 2|x| log2 e overflows.
__device__ __forceinline__ float tanh_sfu(float x)
{
    // Below |x| = 4e-3, tanh(x) = x to within
    // x^3/3 <= 2.2e-8, which also keeps the sign of tiny fields that the
    // difference 1 - 2/(1+e) would round away.
    const float a = fabsf(x) * 2.8853900817779268f;
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(a));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
    const float big = copysignf(fmaf(-2.0f, r, 1.0f), x);
    return fabsf(x) < 4e-3f ? x : big;
}

template <int RT>
struct Vec;
template <>
struct Vec<1> {
    using T = float;
    __device__ static T load(const float* p) { return *p; }
    __device__ static void store(float* p, T v) { *p = v; }
    __device__ static float get(const T& v, int) { return v; }
    __device__ static void set(T& v, int, float x) { v = x; }
};
template <>
struct Vec<2> {
    using T = float2;
    __device__ static T load(const float* p) { return *reinterpret_cast<const float2*>(p); }
    __device__ static void store(float* p, T v) { *reinterpret_cast<float2*>(p) = v; }
    __device__ static float get(const T& v, int k) { return k == 0 ? v.x : v.y; }
    __device__ static void set(T& v, int k, float x) { if (k == 0) v.x = x; else v.y = x; }
};
template <>
struct Vec<4> {
    using T = float4;
    __device__ static T load(const float* p) { return *reinterpret_cast<const float4*>(p); }
    __device__ static void store(float* p, T v) { *reinterpret_cast<float4*>(p) = v; }
    __device__ static float get(const T& v, int k)
    {
        return k == 0 ? v.x : k == 1 ? v.y : k == 2 ? v.z : v.w;
    }
    __device__ static void set(T& v, int k, float x)
    {
        if (k == 0) v.x = x; else if (k == 1) v.y = x; else if (k == 2) v.z = x; else v.w = x;
    }
};

// One coupling: (column, weight). Format 0: (column, float bits) pairs;
// format 1: +-1 words, column | sign << 31; format 2: +-1 halfwords,
// column | sign << 15, staged in shared memory for the whole kernel;
// format 3: the same halfwords read from global memory through L1.
template <int FMT>
struct Entry;
template <>
struct Entry<1> {
    const uint32_t* e;
    __device__ void get(int idx, int& col, float& w) const
    {
        const uint32_t v = __ldg(e + idx);
        col = (int)(v & 0x7fffffffu);
        w = (v >> 31) ? -1.f : 1.f;
    }
};
template <>
struct Entry<0> {
    const int2* e;
    __device__ void get(int idx, int& col, float& w) const
    {
        const int2 v = __ldg(e + idx);
        col = v.x;
        w = __int_as_float(v.y);
    }
};
template <>
struct Entry<2> {
    const uint16_t* e;  // shared memory
    __device__ void get(int idx, int& col, float& w) const
    {
        const uint32_t v = e[idx];
        col = (int)(v & 0x7fffu);
        w = (v >> 15) ? -1.f : 1.f;
    }
};

template <>
struct Entry<3> {
    const uint16_t* e;  // the halfword table in global memory, read through L1
    __device__ void get(int idx, int& col, float& w) const
    {
        const uint32_t v = __ldg(e + idx);
        col = (int)(v & 0x7fffu);
        w = (v >> 15) ? -1.f : 1.f;
    }
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Floats of one CTA's slab of magnetisations in global memory: (n + 1) * rt
// (the dummy row n included), rounded up to 16 bytes so that every slab
// starts on a 16-byte boundary.
__host__ __device__ inline size_t sell_slab_floats(int n, int rt)
{
    return align16((size_t)(n + 1) * rt * sizeof(float)) / sizeof(float);
}

// Per-CTA bookkeeping of the RT replica slots, in shared memory.
template <int RT, int NW>
struct SlotState {
    double T[RT];
    float invT[RT];
    int rep[RT], fresh[RT], done[RT];
    int lvl_sweeps[RT], sweeps[RT], levels[RT], capped[RT], active[RT];
    float dred[NW][RT];
    long long ei[NW][RT];
    double ef[NW][RT];
};

// Run one instance's replica queue on this CTA until the queue is empty and
// every slot has drained. Called by the whole CTA (it contains barriers). The
// slot bookkeeping S may be sized for more slots (RTS) than the job uses.
template <int RT, int NT, int FMT, int DEG = 0, int RTS = RT>
__device__ void run_job(const DevInstance& in, const DevSolve& s, float* m, SlotState<RTS, NT / 32>& S)
{
    static_assert(RT <= RTS, "the slot bookkeeping holds the job's slots");
    constexpr int kThreads = NT;
    constexpr int kWarps = NT / 32;
    using V = Vec<RT>;
    double* const s_T = S.T;
    float* const s_invT = S.invT;
    int* const s_rep = S.rep;
    int* const s_fresh = S.fresh;
    int* const s_done = S.done;
    int* const s_lvl_sweeps = S.lvl_sweeps;
    int* const s_sweeps = S.sweeps;
    int* const s_levels = S.levels;
    int* const s_capped = S.capped;
    int* const s_active = S.active;
    auto& s_dred = S.dred;
    auto& s_ei = S.ei;
    auto& s_ef = S.ef;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = in.n;
    __shared__ int s_last[RT];  // serving ring: this slot finished its job's last replica
    Entry<FMT> ent;
    const int4* slices = in.slices;
    if constexpr (FMT == 0) ent.e = in.sell_gen;
    if constexpr (FMT == 1) ent.e = in.sell_pm1;
    if constexpr (FMT == 3) ent.e = in.sell16;
    if constexpr (FMT == 2) {
        // Stage the slice table and the halfword couplings in shared memory,
        // after the magnetisations; they serve every replica this CTA runs.
        unsigned char* base = reinterpret_cast<unsigned char*>(m);
        int4* ss = reinterpret_cast<int4*>(base + align16((size_t)(n + 1) * RT * sizeof(float)));
        uint16_t* se = reinterpret_cast<uint16_t*>(ss + in.nslices);
        for (int q = tid; q < in.nslices; q += kThreads) ss[q] = __ldg(in.slices + q);
        for (int64_t q = tid; q < in.sell_len; q += kThreads) se[q] = __ldg(in.sell16 + q);
        slices = ss;
        ent.e = se;
        __syncthreads();
    }

    // Each of the RT slots takes replicas from the queue s.tile_rep[0..R) (longest
    // start temperatures first) until it is empty: when a slot's replica ends,
    // the slot is finalised and refilled at once, so no slot idles while work
    // remains.
    if (tid == 0) {
        for (int k = 0; k < RT; ++k) {
            const int q = atomicAdd(s.work_counter, 1);
            const int r = q < s.R ? s.tile_rep[q] : -1;
            s_rep[k] = r;
            s_fresh[k] = r >= 0;
            s_done[k] = 0;
            s_active[k] = 0;
        }
    }
    __syncthreads();

    for (;;) {
        // ---- fresh slots: start state (caller m0 or the draw) and first level --
        bool fresh[RT], any_fresh = false;
#pragma unroll
        for (int k = 0; k < RT; ++k) { fresh[k] = s_fresh[k] != 0; any_fresh |= fresh[k]; }
        if (any_fresh) {
            for (int idx = tid; idx < (n + 1) * RT; idx += kThreads) {
                const int i = idx / RT, k = idx % RT;
                if (!fresh[k]) continue;
                const int r = s_rep[k];
                float v = 0.f;
                if (i < n) {
                    const int o = __ldg(in.new2old + i);
                    v = s.m0 ? __ldg(s.m0 + (size_t)r * n + o) : draw_m0(s.seed, s.stream, r, o);
                }
                m[idx] = v;
            }
            __syncthreads();
            if (tid < RT && fresh[tid]) {
                double T;
                const bool act = sched_first(s, (double)s.t0[s_rep[tid]], &T);
                s_T[tid] = T;
                s_invT[tid] = act ? sched_inv_t(T) : 0.f;
                s_active[tid] = act;
                s_done[tid] = !act;  // no level with T > 0: the result is sign(m0)
                s_levels[tid] = act ? 1 : 0;
                s_lvl_sweeps[tid] = 0;
                s_sweeps[tid] = 0;
                s_capped[tid] = 0;
                s_fresh[tid] = 0;
            }
            __syncthreads();
        }

        // ---- finished slots: sign-round, outputs, exact energy; then refill ----
        bool done[RT], any_done = false;
#pragma unroll
        for (int k = 0; k < RT; ++k) { done[k] = s_done[k] != 0; any_done |= done[k]; }
        if (any_done) {
            long long ei[RT];
            double ef[RT];
            int rep[RT];
#pragma unroll
            for (int k = 0; k < RT; ++k) { ei[k] = 0; ef[k] = 0.0; rep[k] = s_rep[k]; }
            for (int i = tid; i < n; i += kThreads) {
                const int o = __ldg(in.new2old + i);
                const typename V::T mi = V::load(m + i * RT);
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    if (!done[k]) continue;
                    const float mv = V::get(mi, k);
                    s.sigma[(size_t)rep[k] * n + o] = (int8_t)(mv >= 0.f ? 1 : -1);
                    if (s.m_final) s.m_final[(size_t)rep[k] * n + o] = mv;
                }
                const int e0 = __ldg(in.row_ptr + i), e1 = __ldg(in.row_ptr + i + 1);
                for (int e = e0; e < e1; ++e) {
                    const int j = __ldg(in.col + e);
                    if (j <= i) continue;
                    const typename V::T mj = V::load(m + j * RT);
                    if (in.integer) {
                        const int w = (int)__ldg(in.val_i8 + e);
#pragma unroll
                        for (int k = 0; k < RT; ++k)
                            if (done[k])
                                ei[k] += (V::get(mi, k) >= 0.f) == (V::get(mj, k) >= 0.f) ? w : -w;
                    } else {
                        const double w = __ldg(in.val_f64 + e);
#pragma unroll
                        for (int k = 0; k < RT; ++k)
                            if (done[k])
                                ef[k] += (V::get(mi, k) >= 0.f) == (V::get(mj, k) >= 0.f) ? w : -w;
                    }
                }
#pragma unroll
                for (int k = 0; k < RT; ++k) {
                    if (!done[k]) continue;
                    const int si = V::get(mi, k) >= 0.f ? 1 : -1;
                    if (in.integer) {
                        if (in.h) ei[k] += (long long)__ldg(in.h + i) * si;
                    } else if (in.h_f64) {
                        ef[k] += __ldg(in.h_f64 + i) * si;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                const long long a = warp_reduce_strided<1>(ei[k], SumOp());
                const double b = warp_reduce_strided<1>(ef[k], SumOp());
                if (lane == 0) { s_ei[warp][k] = a; s_ef[warp][k] = b; }
            }
            if (s.finished) __threadfence();  // this thread's outputs, before the completion count
            __syncthreads();
            if (tid < RT && done[tid]) {
                const int r = rep[tid];
                long long ti = 0;
                double tf = 0.0;
                for (int w = 0; w < kWarps; ++w) { ti += s_ei[w][tid]; tf += s_ef[w][tid]; }
                s.energy[r] = in.integer ? (double)ti : tf;
                s.energy_i64[r] = in.integer ? ti : 0;
                s.sweeps[r] = s_sweeps[tid];
                s.levels[r] = s_levels[tid];
                s.capped[r] = s_capped[tid];
                if (s.finished) {
                    __threadfence();
                    s_last[tid] = atomicAdd(s.finished, 1) + 1 == s.R;
                }
            }
            __syncthreads();
            if (s.finished) {
                // The CTA that finishes a served job's last replica selects its
                // best replica and tells the host (every CTA fenced its outputs
                // before counting them).
                bool last = false;
#pragma unroll
                for (int k = 0; k < RT; ++k) last |= done[k] && s_last[k] != 0;
                if (last) {
                    __threadfence();
                    best_reduce<kThreads>(s, n, in.integer, s.best_out, s.res);
                    __threadfence_system();
                    __syncthreads();
                    if (tid == 0) *reinterpret_cast<volatile int32_t*>(s.done_flag) = 1;
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < RT; ++k)
                    if (tid == k) s_last[k] = 0;
            }
            if (tid == 0) {
                for (int k = 0; k < RT; ++k) {
                    if (!done[k]) continue;
                    const int q = atomicAdd(s.work_counter, 1);
                    const int r = q < s.R ? s.tile_rep[q] : -1;
                    s_rep[k] = r;
                    s_fresh[k] = r >= 0;
                    s_done[k] = 0;
                }
            }
            __syncthreads();
            continue;
        }

        bool act[RT], any_act = false;
#pragma unroll
        for (int k = 0; k < RT; ++k) { act[k] = s_active[k] != 0; any_act |= act[k]; }
        if (!any_act) break;  // every slot is empty: the queue ran dry

        // ---- one sweep: the levels in order, each a parallel step -------------
        // A thread updates its spin for all RT replicas from one coupling load
        // and RT-wide gathers (dead slots skip only their tanh). When a single
        // slot is left (the queue ran dry) it takes a one-replica path, so a
        // straggler replica's sweep costs what a one-replica sweep costs.
        float invT[RT], dloc[RT];
        int live = 0;
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            invT[k] = s_invT[k];
            dloc[k] = 0.f;
            live |= act[k] ? 1 << k : 0;
        }
        const bool all_live = RT == 1 || __popc(live) > 1;
        const bool lean = live == (1 << RT) - 1 && !in.h;  // uniform over the CTA
        for (int l = 0; l < in.nlev; ++l) {
            const int s0 = __ldg(in.lvl_slice + l), s1 = __ldg(in.lvl_slice + l + 1);
            for (int sl = s0 + warp; sl < s1; sl += kWarps) {
                const int4 d = FMT == 2 ? slices[sl] : __ldg(in.slices + sl);  // row0, rows, degree, offset
                if (lane >= d.y) continue;
                const int i = d.x + lane;
                const float hv = in.h ? __ldg(in.h + i) : 0.f;
                if (all_live) {
                    typename V::T acc;
#pragma unroll
                    for (int k = 0; k < RT; ++k) V::set(acc, k, 0.f);
                    const int deg = DEG > 0 ? DEG : d.z;  // a regular instance's degree is known
#pragma unroll 4
                    for (int q = 0; q < deg; ++q) {
                        int c;
                        float w;
                        ent.get(d.w + 32 * q + lane, c, w);
                        const typename V::T mv = V::load(m + c * RT);
#pragma unroll
                        for (int k = 0; k < RT; ++k)
                            V::set(acc, k, fmaf(w, V::get(mv, k), V::get(acc, k)));
                    }
                    const typename V::T old = V::load(m + i * RT);
                    typename V::T nv;
                    if (lean) {
                        // every slot live, no field: no per-slot test, no add
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
                } else {
#pragma unroll
                    for (int k = 0; k < RT; ++k) {
                        if (!((live >> k) & 1)) continue;
                        float acc = 0.f;
                        const int deg = DEG > 0 ? DEG : d.z;
#pragma unroll 4
                        for (int q = 0; q < deg; ++q) {
                            int c;
                            float w;
                            ent.get(d.w + 32 * q + lane, c, w);
                            acc = fmaf(w, m[c * RT + k], acc);
                        }
                        const float old = m[i * RT + k];
                        const float sn = -tanh_sfu((acc + hv) * invT[k]);
                        dloc[k] = fmaxf(dloc[k], fabsf(sn - old));
                        m[i * RT + k] = sn;
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < RT; ++k) {
            const float v = warp_reduce_strided<1>(dloc[k], MaxOp());
            if (lane == 0) s_dred[warp][k] = v;
        }
        __syncthreads();
        if (warp == 0) {
            // the per-warp maxima of each slot, reduced by warp 0's lanes
            float dk[RT];
#pragma unroll
            for (int k = 0; k < RT; ++k) {
                float v = lane < kWarps ? s_dred[lane][k] : 0.f;
                dk[k] = warp_reduce_strided<1>(v, MaxOp());
            }
            if (lane < RT && s_active[lane]) {
                const int k = lane;
                float dd = dk[0];
#pragma unroll
                for (int q = 1; q < RT; ++q)
                    if (q == k) dd = dk[q];
                int ls = s_lvl_sweeps[k] + 1;
                s_sweeps[k] += 1;
                double T = s_T[k];
                const bool fixed = sched_fixed(s, T);
                const bool level_done = fixed ? ls >= s.fixed_sweeps : (dd <= s.d_min || ls >= s.k_max);
                if (level_done) {
                    if (!fixed && !(dd <= s.d_min)) s_capped[k] += 1;
                    ls = 0;
                    if (sched_advance(s, &T)) {
                        s_T[k] = T;
                        s_levels[k] += 1;
                        s_invT[k] = sched_inv_t(T);
                    } else {
                        s_active[k] = 0;
                        s_done[k] = 1;
                    }
                }
                s_lvl_sweeps[k] = ls;
            }
        }
        __syncthreads();
    }
}
}  // namespace
}  // namespace mars
