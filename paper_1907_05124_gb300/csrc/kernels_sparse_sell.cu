// Sparse MARS descent, fast path: sliced-ELL couplings and on-chip replicas.
//
// Same method and same schedule as kernels_sparse.cu (Section 3, Algorithm 1:
// sequential sweeps reproduced level by level), with a layout built for the
// SM instead of a plain CSR walk:
//
//  * Within a level the runtime sorts spins by degree and cuts them into
//    slices of 32 consecutive new labels (any order inside a level gives the
//    sequential sweep's values, since those spins share no coupling). A
//    slice's couplings are stored slot-major, padded to the slice's largest
//    degree: entry d of row q sits at off + 32*d + q. A warp walks one slice,
//    lane q owns row q, and each of its loads is one coalesced 128-byte line.
//    Padding points at a dummy spin whose magnetisation is held at 0.
//  * +-1 couplings are one 32-bit word: column | sign bit. General weights
//    are a (column, value) pair.
//  * A thread owns one spin for all RT replicas of the tile: one coupling
//    load, one RT-wide shared-memory gather, RT multiply-adds.
//
// The tile's magnetisations m[i*RT + k] live in shared memory for the whole
// descent; the dummy row n is zero. Only the sweeps' parallel steps need a
// block barrier.
#include "device_common.cuh"
#include "mars_internal.h"

#include <algorithm>
#include <cstdlib>

namespace mars {
namespace {

// tanh(x) = sign(x) (1 - 2 / (1 + e^{2|x|})), with e^{2|x|} = 2^{2|x| log2 e}
// from the SFU's ex2.approx and the quotient from its rcp.approx. Absolute
// error below 2.5e-7 over all of R (checked against FP64 tanh through the C
// ABI by the fields-only test); saturates to +-1 when 2|x| log2 e overflows.
__device__ __forceinline__ float tanh_sfu(float x)
{
    // tanh(x) = sign(x) (1 - 2 / (1 + 2^{2|x| log2 e})), SFU ex2 and rcp; below
    // |x| = 1e-3 the odd series x - x^3/3 (error < 2e-16) keeps tiny fields'
    // signs, which the difference 1 - 2/(1+e) would round away.
    const float a = fabsf(x) * 2.8853900817779268f;
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(a));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
    const float big = copysignf(fmaf(-2.0f, r, 1.0f), x);
    const float small = fmaf(x * x, x * -0.333333343f, x);
    return fabsf(x) < 1e-3f ? small : big;
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

// One coupling: (column, weight). PM1 entries pack the sign in bit 31.
template <bool PM1>
struct Entry;
template <>
struct Entry<true> {
    const uint32_t* e;
    __device__ void get(int idx, int& col, float& w) const
    {
        const uint32_t v = __ldg(e + idx);
        col = (int)(v & 0x7fffffffu);
        w = (v >> 31) ? -1.f : 1.f;
    }
};
template <>
struct Entry<false> {
    const int2* e;
    __device__ void get(int idx, int& col, float& w) const
    {
        const int2 v = __ldg(e + idx);
        col = v.x;
        w = __int_as_float(v.y);
    }
};

template <int RT, int NT, bool PM1>
__global__ void __launch_bounds__(NT, 1024 / NT) sparse_sell_kernel(DevInstance in, DevSolve s)
{
    constexpr int kThreads = NT;
    constexpr int kWarps = NT / 32;
    using V = Vec<RT>;
    extern __shared__ __align__(16) float m[];  // (n+1)*RT
    __shared__ double s_T[RT];
    __shared__ float s_invT[RT];
    __shared__ int s_rep[RT], s_fresh[RT], s_done[RT];
    __shared__ int s_lvl_sweeps[RT], s_sweeps[RT], s_levels[RT], s_capped[RT], s_active[RT];
    __shared__ float s_dred[kWarps][RT];
    __shared__ long long s_ei[kWarps][RT];
    __shared__ double s_ef[kWarps][RT];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = in.n;
    Entry<PM1> ent;
    if constexpr (PM1) ent.e = in.sell_pm1; else ent.e = in.sell_gen;

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
                const double T = (double)s.t0[s_rep[tid]] - s.c_step;
                const bool act = T > 0.0;
                s_T[tid] = T;
                s_invT[tid] = act ? (float)(1.0 / T) : 0.f;
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
            }
            __syncthreads();
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
        for (int l = 0; l < in.nlev; ++l) {
            const int s0 = __ldg(in.lvl_slice + l), s1 = __ldg(in.lvl_slice + l + 1);
            for (int sl = s0 + warp; sl < s1; sl += kWarps) {
                const int4 d = __ldg(in.slices + sl);  // row0, rows, degree, offset
                if (lane >= d.y) continue;
                const int i = d.x + lane;
                const float hv = in.h ? __ldg(in.h + i) : 0.f;
                if (all_live) {
                    typename V::T acc;
#pragma unroll
                    for (int k = 0; k < RT; ++k) V::set(acc, k, 0.f);
#pragma unroll 4
                    for (int q = 0; q < d.z; ++q) {
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
                    V::store(m + i * RT, nv);
                } else {
#pragma unroll
                    for (int k = 0; k < RT; ++k) {
                        if (!((live >> k) & 1)) continue;
                        float acc = 0.f;
#pragma unroll 4
                        for (int q = 0; q < d.z; ++q) {
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
        if (tid < RT && s_active[tid]) {
            float dd = 0.f;
#pragma unroll 8
            for (int w = 0; w < kWarps; ++w) dd = fmaxf(dd, s_dred[w][tid]);
            int ls = s_lvl_sweeps[tid] + 1;
            s_sweeps[tid] += 1;
            const bool level_done = s.fixed_sweeps > 0 ? ls >= s.fixed_sweeps
                                                       : (dd <= s.d_min || ls >= s.k_max);
            if (level_done) {
                if (s.fixed_sweeps == 0 && !(dd <= s.d_min)) s_capped[tid] += 1;
                const double T = s_T[tid] - s.c_step;
                s_T[tid] = T;
                ls = 0;
                if (T > 0.0) {
                    s_levels[tid] += 1;
                    s_invT[tid] = (float)(1.0 / T);
                } else {
                    s_active[tid] = 0;
                    s_done[tid] = 1;
                }
            }
            s_lvl_sweeps[tid] = ls;
        }
        __syncthreads();
    }
}

template <int RT, int NT>
const void* pick_nt(bool pm1)
{
    return pm1 ? (const void*)sparse_sell_kernel<RT, NT, true> : (const void*)sparse_sell_kernel<RT, NT, false>;
}

const void* pick(int rt, int nt, bool pm1)
{
    if (nt == 512) {
        switch (rt) {
        case 1: return pick_nt<1, 512>(pm1);
        case 2: return pick_nt<2, 512>(pm1);
        case 4: return pick_nt<4, 512>(pm1);
        }
    } else if (nt == 1024) {
        switch (rt) {
        case 1: return pick_nt<1, 1024>(pm1);
        case 2: return pick_nt<2, 1024>(pm1);
        case 4: return pick_nt<4, 1024>(pm1);
        }
    }
    return nullptr;
}

int env_int(const char* name, int dflt)
{
    const char* v = std::getenv(name);
    return v && *v ? std::atoi(v) : dflt;
}

}  // namespace

// Launch shape: replica slots per CTA (RT) and threads per CTA. A GB300
// sweep of the six shapes on the 2-D L=100 lattice, R=1024 (spin-updates/s):
// RT=2 with 1024 threads 3.46e11; RT=1/1024 2.63e11; RT=4/1024 2.64e11;
// the 512-thread shapes 2.0-2.2e11. Wider CTAs give a lone replica's sweep
// more threads; two slots amortise the coupling loads without the 4-wide
// tail. MARS_SELL_RT / MARS_SELL_THREADS override the choice for tuning.
bool plan_sparse_sell(const DevInstance& in, int R, int device, SparsePlan* p)
{
    if (!in.slices || (!in.sell_pm1 && !in.sell_gen)) return false;
    int sms = 1, optin = 48 * 1024;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t budget = (size_t)optin - 12 * 1024;  // static shared memory and slack
    int rt = env_int("MARS_SELL_RT", 2);
    int nt = env_int("MARS_SELL_THREADS", 1024);
    if (rt != 1 && rt != 2 && rt != 4) rt = 1;
    if (nt != 512 && nt != 1024) nt = 512;
    while (rt > 1 && (size_t)(in.n + 1) * rt * sizeof(float) > budget) rt /= 2;
    if ((size_t)(in.n + 1) * rt * sizeof(float) > budget) return false;
    p->rt = rt;
    p->onchip = 1;
    p->threads = nt;
    p->smem = (size_t)(in.n + 1) * rt * sizeof(float);
    p->sell = 1;
    const void* k = pick(rt, nt, in.sell_pm1 != nullptr);
    if (!k) return false;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, p->smem);
    if (per_sm < 1) per_sm = 1;
    const int ntiles = (R + rt - 1) / rt;
    p->grid = std::max(1, std::min(ntiles, sms * per_sm));
    p->scratch_floats = 0;
    return true;
}

cudaError_t launch_sparse_sell(const DevInstance& in, const DevSolve& s, const SparsePlan& p,
                               cudaStream_t st)
{
    const void* k = pick(p.rt, p.threads, in.sell_pm1 != nullptr);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    DevInstance a = in;
    DevSolve b = s;
    void* args[] = {&a, &b};
    return cudaLaunchKernel(k, dim3(p.grid), dim3(p.threads), args, p.smem, st);
}

}  // namespace mars
