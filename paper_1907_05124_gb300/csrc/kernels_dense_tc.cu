// Dense MARS descent with tcgen05 tensor cores (BF16 operands, FP32 fields).
//
// A sweep visits the spins sequentially (Section 3, Algorithm 1 with the
// per-spin update of the GPU text). For dense J every spin couples to every
// other, so the sweep is cut into panels of 128 consecutive spins and each
// panel p does two things, exactly reproducing the sequential sweep:
//
//   1. G = J[p, :] S^T over all active replicas, one tensor-core GEMM
//      (panel_gemm_kernel): S holds the newest values of panels < p and the
//      old values of panels >= p, in BF16; split-K partials in FP32.
//   2. The panel's spins in order (panel_chain_kernel, one warp per replica):
//      Phi_a = G_a + sum_{b in p, b < a} J_ab (s_b_new - s_b_used_in_G) + h_a,
//      s_a = -tanh(Phi_a / T); each new s_a is folded into the remaining
//      fields of the panel from the FP32 diagonal block of J.
//
// The GEMM is the O(n^2 R) part of the sweep; the chain adds O(n * 128 * R).
// Replicas live in slots ordered by start temperature (longest first), so the
// active ones form a prefix and the GEMM skips tiles past it.
#include "device_common.cuh"
#include "mars_internal.h"
#include "tc_primitives.cuh"

#include <cuda_bf16.h>

namespace mars {
namespace {

constexpr int kBM = 128;     // panel rows = MMA M
constexpr int kBK = 64;      // K per pipeline stage: one 128-byte swizzle row of BF16
constexpr int kStages = 4;
constexpr int kChainWarps = 8;

__device__ __forceinline__ float tanh_sfu(float x)
{
    // tanh(x) = sign(x) (1 - 2 / (1 + 2^{2|x| log2 e})), SFU ex2 and rcp
    // (absolute error ~6e-8). Below |x| = 4e-3, tanh(x) = x to within
    // x^3/3 <= 2.2e-8, which also keeps the sign of tiny fields that the
    // difference 1 - 2/(1+e) would round away.
    const float a = fabsf(x) * 2.8853900817779268f;
    float e, r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(a));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
    const float big = copysignf(fmaf(-2.0f, r, 1.0f), x);
    return fabsf(x) < 4e-3f ? x : big;
}

template <int BN>
struct GemmSmem {
    static constexpr uint32_t kA = kBM * kBK * 2;
    static constexpr uint32_t kB = BN * kBK * 2;
    static constexpr size_t kBytes = 1024 + kStages * (kA + kB) + (2 * kStages + 1) * 8 + 16;
};

// G_part[split][slot][a] = sum over this split's K range of J[p0 + a][k] S[slot][k].
template <int BN>
__global__ void __launch_bounds__(128, 1)
    panel_gemm_kernel(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmS,
                      TcPanel g)
{
    using L = GemmSmem<BN>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;
    unsigned char* sB = smem + kStages * L::kA;
    uint64_t* full = (uint64_t*)(sB + kStages * L::kB);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);

    const int n0 = blockIdx.x * BN;
    if (n0 >= *g.active_prefix) return;  // whole CTA, before any barrier
    const int split = blockIdx.y;
    const int kb0 = split * g.kblocks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        tc::tma_prefetch_desc(&tmJ);
        tc::tma_prefetch_desc(&tmS);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, BN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer: stage s is free once the MMAs that read it completed.
        for (int kb = 0; kb < g.kblocks; ++kb) {
            const int s = kb % kStages;
            if (kb >= kStages && !tc::mbar_wait(&empty[s], ((kb / kStages) - 1) & 1, g.err)) break;
            tc::mbar_arrive_expect_tx(&full[s], L::kA + L::kB);
            tc::tma_load_2d(sA + s * L::kA, &tmJ, &full[s], (kb0 + kb) * kBK, g.p0);
            tc::tma_load_2d(sB + s * L::kB, &tmS, &full[s], (kb0 + kb) * kBK, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: four K=16 steps per stage, accumulator in TMEM.
        constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, BN);
        for (int kb = 0; kb < g.kblocks; ++kb) {
            const int s = kb % kStages;
            if (!tc::mbar_wait(&full[s], (kb / kStages) & 1, g.err)) break;
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_addr(sA + s * L::kA), b0 = tc::smem_addr(sB + s * L::kB);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
                tc::mma_bf16(tmem, tc::smem_desc_sw128(a0 + k * 32), tc::smem_desc_sw128(b0 + k * 32),
                             idesc, (kb | k) != 0);
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(done);
    }
    __syncwarp();

    // Epilogue: TMEM lane = panel row, columns = replica slots.
    const bool ok = tc::mbar_wait(done, 0, g.err);
    tc::tc_fence_after();
    const int row = warp * 32 + lane;
    float* dst = g.G + ((size_t)split * g.R_pad + n0) * kBM + row;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tc::tmem_ld_32cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (ok) {
#pragma unroll
            for (int j = 0; j < 32; ++j) dst[(size_t)(c0 + j) * kBM] = v[j];
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, BN);
}

// Compensated accumulate: (s, c) += a * b with the product's and the sum's
// rounding errors carried in c (TwoProduct by FMA, TwoSum; Ogita, Rump,
// Oishi 2005). Used where a panel's field is assembled from its split-K
// partial sums and the field h. The in-panel corrections use plain FMAs:
// beside a BF16 GEMM their FP32 rounding is immaterial.
__device__ __forceinline__ void acc2(float& s, float& c, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
}

// One warp per replica slot: the panel's 128 spins in sequence.
// Per spin of the panel, what every lane of a replica's warp reads at that
// spin's step: the low part of its field, its old FP32 and BF16 values and
// J[a-1][a], the coupling to the spin updated just before it.
struct ChainSpin {
    float gc, s_old, s_old_bf, j_prev;
};
constexpr int kMaxSplit = 8;
constexpr int kChainSmem = kBM * kBM * (int)sizeof(float) + kChainWarps * kBM * (int)sizeof(ChainSpin);

// The chain with one step of lookahead. Every lane computes the update of the
// current spin a itself, from g_a as it stood before the last change
// (broadcast during the previous step) plus J[a-1][a] * delta_{a-1}; the
// lanes that own the panel's other spins fold delta_a into their fields. The
// broadcast of g_{a+1} thus overlaps the update of spin a, and a step's
// critical path is one FMA, the tanh and one subtraction, with no shuffle
// and no divergence. Operations and their order are those of the plain
// chain (the owner of spin a would apply the same FMAs), so the fields are
// bit-identical to it.
__global__ void __launch_bounds__(kChainWarps * 32) panel_chain_kernel(TcState t, int p)
{
    extern __shared__ __align__(16) float Jb[];  // FP32 diagonal block of J (symmetric), 64 KB
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float* src = t.Jdiag + (size_t)p * kBM * kBM;
    for (int i = threadIdx.x; i < kBM * kBM / 4; i += blockDim.x)
        reinterpret_cast<float4*>(Jb)[i] = __ldg(reinterpret_cast<const float4*>(src) + i);
    ChainSpin* cs = reinterpret_cast<ChainSpin*>(Jb + kBM * kBM) + warp * kBM;
    __syncthreads();
    const int slot = blockIdx.x * kChainWarps + warp;
    if (slot >= t.R || !t.active[slot]) return;
    const int p0 = p * kBM;
    const float invT = t.invT[slot];
    // Split-K partial fields: every load first, then the compensated sum in
    // split order, then h.
    float gp[kMaxSplit][4];
#pragma unroll
    for (int sp = 0; sp < kMaxSplit; ++sp)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            gp[sp][q] = sp < t.splitk ? t.G[((size_t)sp * t.R_pad + slot) * kBM + lane + 32 * q] : 0.f;
    float g[4], sf[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int a = lane + 32 * q;
        float acc = 0.f, accc = 0.f;
#pragma unroll
        for (int sp = 0; sp < kMaxSplit; ++sp)
            if (sp < t.splitk) acc2(acc, accc, gp[sp][q], 1.0f);
        if (t.h && p0 + a < t.n) acc2(acc, accc, __ldg(t.h + p0 + a), 1.0f);
        g[q] = acc;
        const size_t idx = (size_t)slot * t.n_pad + p0 + a;
        sf[q] = t.S[idx];
        cs[a] = ChainSpin{accc, sf[q], __bfloat162float(t.Sb[idx]), a > 0 ? Jb[(a - 1) * kBM + a] : 0.f};
    }
    __syncwarp();
    float ghat = __shfl_sync(0xffffffffu, g[0], 0);
    // -0 * 0 + ghat == ghat for every ghat, so the first step's FMA is exact
    float dprev = -0.f, dloc = 0.f;
#pragma unroll
    for (int qa = 0; qa < 4; ++qa) {
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
            const int a = qa * 32 + l;
            const ChainSpin c = cs[a];
            const float x = fmaf(c.j_prev, dprev, ghat);
            const float sn = -tanh_sfu((x + c.gc) * invT);
            dloc = fmaxf(dloc, fabsf(sn - c.s_old));
            const float delta = sn - c.s_old_bf;
            if (lane == l) sf[qa] = sn;
            // g_{a+1} before delta_a reaches it; its owner applies delta_a below
            const float gsrc = l < 31 ? g[qa] : g[qa < 3 ? qa + 1 : 3];
            ghat = __shfl_sync(0xffffffffu, gsrc, (l + 1) & 31);
            const float* Jrow = Jb + a * kBM;
#pragma unroll
            for (int q = qa; q < 4; ++q) g[q] = fmaf(Jrow[lane + 32 * q], delta, g[q]);
            dprev = delta;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int a = lane + 32 * q;
        if (p0 + a < t.n) {
            const size_t idx = (size_t)slot * t.n_pad + p0 + a;
            t.S[idx] = sf[q];
            t.Sb[idx] = __float2bfloat16_rn(sf[q]);
        }
    }
    // every lane computed every spin's change, so dloc is the warp's maximum
    if (lane == 0) t.d[slot] = fmaxf(t.d[slot], dloc);
}

// Start states in slot order: slot j holds replica rep[j].
__global__ void tc_init_kernel(TcState t)
{
    const size_t total = (size_t)t.R * t.n_pad;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int slot = (int)(idx / t.n_pad), a = (int)(idx % t.n_pad);
        const int r = t.rep[slot];
        float v = 0.f;
        if (a < t.n) {
            const int o = __ldg(t.new2old + a);
            v = t.m0 ? __ldg(t.m0 + (size_t)r * t.n + o) : draw_m0(t.seed, t.stream, r, o);
        }
        t.S[idx] = v;
        t.Sb[idx] = __float2bfloat16_rn(v);
    }
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < t.R; slot += gridDim.x * blockDim.x) {
        const double T = (double)t.t0[t.rep[slot]] - t.c_step;
        const bool act = T > 0.0;
        t.T[slot] = T;
        t.invT[slot] = act ? (float)(1.0 / T) : 0.f;
        t.active[slot] = act;
        t.levels[slot] = act ? 1 : 0;
        t.lvl_sweeps[slot] = 0;
        t.sweeps[slot] = 0;
        t.capped[slot] = 0;
        t.d[slot] = 0.f;
    }
}

// End of a sweep: the stopping rule and the level schedule per slot.
__global__ void tc_advance_kernel(TcState t)
{
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < t.R; slot += gridDim.x * blockDim.x) {
        if (!t.active[slot]) continue;
        const float dd = t.d[slot];
        t.d[slot] = 0.f;
        const int ls = t.lvl_sweeps[slot] + 1;
        t.sweeps[slot] += 1;
        const bool level_done = t.fixed_sweeps > 0 ? ls >= t.fixed_sweeps
                                                   : (dd <= t.d_min || ls >= t.k_max);
        if (level_done) {
            if (t.fixed_sweeps == 0 && !(dd <= t.d_min)) t.capped[slot] += 1;
            const double T = t.T[slot] - t.c_step;
            t.T[slot] = T;
            t.lvl_sweeps[slot] = 0;
            if (T > 0.0) {
                t.levels[slot] += 1;
                t.invT[slot] = (float)(1.0 / T);
            } else {
                t.active[slot] = 0;
            }
        } else {
            t.lvl_sweeps[slot] = ls;
        }
    }
}

// Active prefix (one past the last active slot) and active count.
__global__ void tc_prefix_kernel(TcState t)
{
    __shared__ int s_max, s_cnt;
    if (threadIdx.x == 0) { s_max = 0; s_cnt = 0; }
    __syncthreads();
    int mx = 0, cnt = 0;
    for (int slot = threadIdx.x; slot < t.R; slot += blockDim.x)
        if (t.active[slot]) { mx = max(mx, slot + 1); ++cnt; }
    atomicMax(&s_max, mx);
    atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) { t.counters[0] = s_max; t.counters[1] = s_cnt; }
}

// Sign-round, outputs in caller labels and exact energy, one CTA per slot.
__global__ void __launch_bounds__(256) tc_finalize_kernel(TcState t, DevInstance in, DevSolve s)
{
    __shared__ long long s_i[8];
    __shared__ double s_f[8];
    const int slot = blockIdx.x;
    if (slot >= t.R) return;
    const int r = t.rep[slot], n = t.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* m = t.S + (size_t)slot * t.n_pad;
    long long ei = 0;
    double ef = 0.0;
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        const int sa = m[a] >= 0.f ? 1 : -1;
        const int o = __ldg(in.new2old + a);
        s.sigma[(size_t)r * n + o] = (int8_t)sa;
        if (s.m_final) s.m_final[(size_t)r * n + o] = m[a];
        if (in.integer) {
            const int8_t* row = in.J_i8 + (size_t)a * n;
            int acc = 0;
            for (int b = a + 1; b < n; ++b) acc += (int)row[b] * (m[b] >= 0.f ? 1 : -1);
            ei += (long long)acc * sa;
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
    if (lane == 0) { s_i[warp] = ei; s_f[warp] = ef; }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long ti = 0;
        double tf = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) { ti += s_i[w]; tf += s_f[w]; }
        s.energy[r] = in.integer ? (double)ti : tf;
        s.energy_i64[r] = in.integer ? ti : 0;
        s.sweeps[r] = t.sweeps[slot];
        s.levels[r] = t.levels[slot];
        s.capped[r] = t.capped[slot];
    }
}

__global__ void tc_export_kernel(TcState t, DevInstance in, float* m_out, double* t_last)
{
    const size_t total = (size_t)t.R * t.n;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int slot = (int)(idx / t.n), a = (int)(idx % t.n);
        const int r = t.rep[slot];
        m_out[(size_t)r * t.n + __ldg(in.new2old + a)] = t.S[(size_t)slot * t.n_pad + a];
    }
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < t.R; slot += gridDim.x * blockDim.x)
        t_last[t.rep[slot]] = t.levels[slot] > 0 ? t.T[slot] + t.c_step : 0.0;
}

}  // namespace

cudaError_t launch_tc_export(const TcState& t, const DevInstance& in, float* m_out, double* t_last,
                             cudaStream_t st)
{
    tc_export_kernel<<<1024, 256, 0, st>>>(t, in, m_out, t_last);
    return cudaGetLastError();
}

size_t tc_gemm_smem(int bn) { return bn == 64 ? GemmSmem<64>::kBytes : GemmSmem<128>::kBytes; }

cudaError_t launch_tc_panel_gemm(const CUtensorMap& tmJ, const CUtensorMap& tmS, const TcPanel& g,
                                 int bn, int n_tiles, int splitk, cudaStream_t st)
{
    const void* k = bn == 64 ? (const void*)panel_gemm_kernel<64> : (const void*)panel_gemm_kernel<128>;
    const size_t smem = tc_gemm_smem(bn);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    CUtensorMap a = tmJ, b = tmS;
    TcPanel c = g;
    void* args[] = {&a, &b, &c};
    return cudaLaunchKernel(k, dim3(n_tiles, splitk), dim3(128), args, smem, st);
}

cudaError_t launch_tc_chain(const TcState& t, int p, cudaStream_t st)
{
    if (t.splitk < 1 || t.splitk > kMaxSplit) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(panel_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kChainSmem);
    if (e != cudaSuccess) return e;
    panel_chain_kernel<<<(t.R + kChainWarps - 1) / kChainWarps, kChainWarps * 32, kChainSmem, st>>>(t, p);
    return cudaGetLastError();
}

cudaError_t launch_tc_init(const TcState& t, cudaStream_t st)
{
    tc_init_kernel<<<1024, 256, 0, st>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_tc_advance(const TcState& t, cudaStream_t st)
{
    tc_advance_kernel<<<(t.R + 255) / 256, 256, 0, st>>>(t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tc_prefix_kernel<<<1, 1024, 0, st>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_tc_prefix(const TcState& t, cudaStream_t st)
{
    tc_prefix_kernel<<<1, 1024, 0, st>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_tc_finalize(const TcState& t, const DevInstance& in, const DevSolve& s,
                               cudaStream_t st)
{
    tc_finalize_kernel<<<t.R, 256, 0, st>>>(t, in, s);
    return cudaGetLastError();
}

}  // namespace mars
