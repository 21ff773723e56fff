// Dense MARS descent with tcgen05 tensor cores (BF16 or E4M3 operands, FP32
// fields).
//
// A sweep visits the spins sequentially (Section 3, Algorithm 1 with the
// per-spin update of the GPU text). For dense J every spin couples to every
// other, so the sweep is cut into panels of 128 consecutive spins and each
// panel p does two things, reproducing the sequential sweep:
//
//   1. G = J[p, :] S^T over all active replicas, one tensor-core GEMM
//      (panel_gemm_kernel): S holds the newest values of panels < p and the
//      old values of panels >= p, in BF16 (or E4M3); split-K partials in FP32.
//   2. The panel's spins in order (panel_chain_kernel, 1, 2 or 4 replicas per
//      warp): Phi_a = G_a + sum_{b in p, b < a} J_ab (s_b_new - s_b_used_in_G)
//      + h_a, s_a = -tanh(Phi_a / T); each new s_a is folded into the
//      remaining fields of the panel from the FP32 diagonal block of J.
//
// Two schedules reorganise the GEMMs. With the overlap, panel p+1's GEMM
// leaves panel p's K blocks out and runs beside chain p on a second stream;
// with panel pairs (pair_gemm_kernel), one GEMM computes panels 2q and 2q+1.
// Either way the left-out block reaches the next panel through the chain, in
// FP32 from J[p][p+1].
//
// The GEMM is the O(n^2 R) part of the sweep; the chain adds O(n * 128 * R).
// Replicas live in slots ordered by start temperature (longest first), so the
// active ones form a prefix and the GEMM skips tiles past it.
#include "device_common.cuh"
#include "mars_internal.h"
#include "schedule.cuh"
#include "tc_primitives.cuh"

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cstdlib>

namespace mars {
namespace {

constexpr int kBM = 128;     // panel rows = MMA M
constexpr int kBK = 64;      // K per pipeline stage: one 128-byte swizzle row of BF16 (128 of E4M3)
#ifndef MARS_GEMM_STAGES
#define MARS_GEMM_STAGES 4
#endif
constexpr int kStages = MARS_GEMM_STAGES;  // TMA pipeline depth of the panel GEMM
constexpr int kChainWarps = 8;

__device__ __forceinline__ float tanh_sfu(float x)
{
    // tanh(x) = sign(x) (1 - 2 / (1 + 2^{2|x| log2 e})), SFU ex2 and rcp;
    // absolute error at most 2.5e-7 against FP64 tanh (the bound the
    // fields-only test through the C ABI holds it to). Below |x| = 4e-3, tanh(x) = x to within
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

// One (tile, split) item of a panel GEMM, on the CTA's warps 0..3:
// G_part[split][slot][a] = sum over this split's K range of J[p0 + a][k] S[slot][k]
// for the BN replica slots from n0. Warp 0's lane 0 is the TMA producer, warp
// 1's lane 0 issues the MMAs (accumulator in TMEM), and warps 0..3 run the
// epilogue (TMEM lane = panel row); other warps only count. `it` is the
// number of stage-ring uses before this item (its phases continue across
// items) and `commits` the number of earlier items that issued MMAs (the done
// barrier's phase). Returns the stage uses after this item; *committed says
// whether it issued MMAs. A split whose K blocks were all left out writes
// zeros. FP8: E4M3 operands (kind::f8f6f4); a stage's 128-byte rows then hold
// 128 K values instead of 64, and a 128-spin panel is one K block instead of two.
template <int BN, bool FP8>
__device__ __forceinline__ int gemm_item(const CUtensorMap* tmJ, const CUtensorMap* tmS, const TcPanel& g,
                                         int n0, int split, unsigned char* sA, unsigned char* sB,
                                         uint64_t* full, uint64_t* empty, uint64_t* done, uint32_t tmem,
                                         int it0, int commits, bool* committed)
{
    using L = GemmSmem<BN>;
    constexpr int kKE = FP8 ? 2 * kBK : kBK;  // K values per stage
    constexpr int kSkipN = kBM / kKE;         // K blocks of one panel
    const int kb0 = split * g.kblocks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // K blocks [skip_kb, skip_kb + kSkipN), one 128-spin panel, may be left
    // out; every thread counts the blocks this split keeps.
    auto skipped = [&](int kb) {
        return g.skip_kb >= 0 && kb0 + kb >= g.skip_kb && kb0 + kb < g.skip_kb + kSkipN;
    };
    int issued = 0;
    for (int kb = 0; kb < g.kblocks; ++kb) issued += skipped(kb) ? 0 : 1;

    if (issued > 0 && warp == 0 && lane == 0) {
        // TMA producer: stage s is free once the MMAs that read it completed.
        int it = it0;
        for (int kb = 0; kb < g.kblocks; ++kb) {
            if (skipped(kb)) continue;
            const int s = it % kStages;
            if (it >= kStages && !tc::mbar_wait(&empty[s], ((it / kStages) - 1) & 1, g.err)) break;
            tc::mbar_arrive_expect_tx(&full[s], L::kA + L::kB);
            tc::tma_load_2d(sA + s * L::kA, tmJ, &full[s], (kb0 + kb) * kKE, g.p0);
            tc::tma_load_2d(sB + s * L::kB, tmS, &full[s], (kb0 + kb) * kKE, n0);
            ++it;
        }
    } else if (issued > 0 && warp == 1 && lane == 0) {
        // MMA issuer: four 32-byte K steps per stage (K = 16 BF16 or 32 E4M3),
        // accumulator in TMEM; the item's first MMA overwrites it.
        constexpr uint32_t idesc = FP8 ? tc::idesc_e4m3_f32(kBM, BN) : tc::idesc_bf16_f32(kBM, BN);
        int it = it0;
        for (int kb = 0; kb < g.kblocks; ++kb) {
            if (skipped(kb)) continue;
            const int s = it % kStages;
            if (!tc::mbar_wait(&full[s], (it / kStages) & 1, g.err)) break;
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_addr(sA + s * L::kA), b0 = tc::smem_addr(sB + s * L::kB);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t acc = ((it - it0) | k) != 0;
                if (FP8)
                    tc::mma_e4m3(tmem, tc::smem_desc_sw128(a0 + k * 32), tc::smem_desc_sw128(b0 + k * 32),
                                 idesc, acc);
                else
                    tc::mma_bf16(tmem, tc::smem_desc_sw128(a0 + k * 32), tc::smem_desc_sw128(b0 + k * 32),
                                 idesc, acc);
            }
            tc::mma_commit(&empty[s]);
            ++it;
        }
        tc::mma_commit(done);
    }
    __syncwarp();

    if (warp < 4) {
        const bool ok = issued > 0 ? tc::mbar_wait(done, (uint32_t)commits & 1u, g.err) : true;
        tc::tc_fence_after();
        const int row = warp * 32 + lane;
        float* dst = g.G + ((size_t)split * g.R_pad + n0) * kBM + row;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            float v[32];
            if (issued > 0) {
                tc::tmem_ld_32cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.f;
            }
            if (ok) {
#pragma unroll
                for (int j = 0; j < 32; ++j) dst[(size_t)(c0 + j) * kBM] = v[j];
            }
        }
    }
    *committed = issued > 0;
    return it0 + issued;
}

// The panel GEMM as its own launch: a grid of (replica tile, split) items
// over the active prefix.
template <int BN, bool FP8>
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

    tc::pdl_wait();  // the previous kernel's spins and active prefix
    tc::pdl_launch_dependents();
    const int n0 = blockIdx.x * BN;
    if (n0 >= *g.active_prefix) return;  // whole CTA, before any barrier
    const int warp = threadIdx.x >> 5;
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
    bool committed;
    gemm_item<BN, FP8>(&tmJ, &tmS, g, n0, blockIdx.y, sA, sB, full, empty, done, tmem, 0, 0, &committed);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, BN);
}

template <int BN>
struct PairSmem {
    static constexpr uint32_t kA = kBM * kBK * 2;     // one 128-row A tile
    static constexpr uint32_t kB = BN * kBK * 2;
    static constexpr uint32_t kStage = 2 * kA + kB;   // both panels' rows and one B tile
    static constexpr size_t kBytes = 1024 + kStages * kStage + (2 * kStages + 1) * 8 + 16;
};

// Two panels' fields from one pass over K. Accumulator 0 (TMEM columns
// [0, BN)) takes panel q's rows (first row g.p0) over every K block;
// accumulator 1 (columns [BN, 2 BN)) takes panel q+1's rows over every K
// block but panel q's own (g.skip_kb and on), since panel q's new spins reach
// panel q+1 through its chain in FP32. Both read the same B tile, so the
// magnetisations are streamed once per pair of panels instead of once per
// panel. Partials go to g.G (panel q) and g.G1 (panel q+1).
template <int BN, bool FP8>
__global__ void __launch_bounds__(128, 1)
    pair_gemm_kernel(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmS,
                     TcPanel g)
{
    using L = PairSmem<BN>;
    constexpr int kKE = FP8 ? 2 * kBK : kBK;
    constexpr int kSkipN = kBM / kKE;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + kStages * L::kStage);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);

    tc::pdl_wait();  // the previous kernel's spins and active prefix
    tc::pdl_launch_dependents();
    const int n0 = blockIdx.x * BN;
    if (n0 >= *g.active_prefix) return;  // whole CTA, before any barrier
    const int split = blockIdx.y;
    const int kb0 = split * g.kblocks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto own = [&](int kb) { return kb0 + kb >= g.skip_kb && kb0 + kb < g.skip_kb + kSkipN; };
    int issued1 = 0;  // K blocks accumulator 1 takes (every thread counts them)
    for (int kb = 0; kb < g.kblocks; ++kb) issued1 += own(kb) ? 0 : 1;

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
    if (warp == 0) tc::tmem_alloc(tmem_slot, 2 * BN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer: panel q+1's A tile is not loaded for panel q's K blocks.
        for (int kb = 0; kb < g.kblocks; ++kb) {
            const int s = kb % kStages;
            if (kb >= kStages && !tc::mbar_wait(&empty[s], ((kb / kStages) - 1) & 1, g.err)) break;
            unsigned char* st = smem + s * L::kStage;
            const bool both = !own(kb);
            tc::mbar_arrive_expect_tx(&full[s], L::kA + L::kB + (both ? L::kA : 0u));
            tc::tma_load_2d(st, &tmJ, &full[s], (kb0 + kb) * kKE, g.p0);
            if (both) tc::tma_load_2d(st + L::kA, &tmJ, &full[s], (kb0 + kb) * kKE, g.p0 + kBM);
            tc::tma_load_2d(st + 2 * L::kA, &tmS, &full[s], (kb0 + kb) * kKE, n0);
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = FP8 ? tc::idesc_e4m3_f32(kBM, BN) : tc::idesc_bf16_f32(kBM, BN);
        int it1 = 0;
        for (int kb = 0; kb < g.kblocks; ++kb) {
            const int s = kb % kStages;
            if (!tc::mbar_wait(&full[s], (kb / kStages) & 1, g.err)) break;
            tc::tc_fence_after();
            const uint32_t a0 = tc::smem_addr(smem + s * L::kStage);
            const uint32_t a1 = a0 + L::kA, b0 = a0 + 2 * L::kA;
            const bool both = !own(kb);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t bd = tc::smem_desc_sw128(b0 + k * 32);
                if (FP8) {
                    tc::mma_e4m3(tmem, tc::smem_desc_sw128(a0 + k * 32), bd, idesc, (kb | k) != 0);
                    if (both)
                        tc::mma_e4m3(tmem + BN, tc::smem_desc_sw128(a1 + k * 32), bd, idesc, (it1 | k) != 0);
                } else {
                    tc::mma_bf16(tmem, tc::smem_desc_sw128(a0 + k * 32), bd, idesc, (kb | k) != 0);
                    if (both)
                        tc::mma_bf16(tmem + BN, tc::smem_desc_sw128(a1 + k * 32), bd, idesc, (it1 | k) != 0);
                }
            }
            it1 += both ? 1 : 0;
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(done);
    }
    __syncwarp();

    const bool ok = tc::mbar_wait(done, 0, g.err);
    tc::tc_fence_after();
    const int row = warp * 32 + lane;
    float* dst0 = g.G + ((size_t)split * g.R_pad + n0) * kBM + row;
    float* dst1 = g.G1 + ((size_t)split * g.R_pad + n0) * kBM + row;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tc::tmem_ld_32cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (ok) {
#pragma unroll
            for (int j = 0; j < 32; ++j) dst0[(size_t)(c0 + j) * kBM] = v[j];
        }
        if (issued1 > 0) {
            tc::tmem_ld_32cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(BN + c0), v);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0.f;
        }
        if (ok) {
#pragma unroll
            for (int j = 0; j < 32; ++j) dst1[(size_t)(c0 + j) * kBM] = v[j];
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * BN);
}

// Per spin of the panel and replica: its field (the split-K partials in
// split order, the previous panel's FP32 part and h, summed in FP32: beside
// the BF16 products their rounding is immaterial, and BF16-exact operands
// sum exactly) and its old FP32 and BF16 values.
struct ChainSpin {
    float g, s_old, s_old_bf, unused;
};

// Shared memory of the chain: the FP32 block J[p][p] (and J[p][p+1] when the
// chain feeds the next panel), the CTA's ChainSpin rows and the mbarrier of
// the bulk copies.
template <int RPW, bool NEXT, int CW = kChainWarps>
struct ChainSmem {
    static constexpr int kJ = kBM * kBM * (int)sizeof(float);
    static constexpr int kBlocks = NEXT ? 2 : 1;
    static constexpr int kCs = CW * RPW * kBM * (int)sizeof(ChainSpin);
    static constexpr int kBytes = kBlocks * kJ + kCs + 16;
};

// The panel's spins in sequence for RPW replicas per warp, 32/RPW lanes per
// replica; lane j of a replica's group owns the spins j + (32/RPW) q.
//
// Prologue: one thread starts bulk copies of the J blocks; meanwhile every
// thread issues all loads for its RPW four-spin pieces of the CTA's fields
// (at most kChainMaxSplit / RPW split-K partials each) in one round trip.
//
// One step of lookahead: every lane of the group computes the update of the
// current spin a itself, from g_a as it stood before the last change
// (broadcast during the previous step) plus J[a-1][a] * delta_{a-1}, and the
// owners fold delta_a into the fields of the panel's later spins. The
// broadcast of g_{a+1} thus overlaps the update of spin a, and with the
// constants of the step folded (below) a step's critical path is one FMA,
// ex2, one add, rcp, one FMA and two selects, with no divergence. The
// owners' FMAs are those of the plain chain in its order; the folding
// reassociates the last term of each field, an FP32 rounding difference.
// Every replicas-per-warp choice computes bit-identical results.
//
// NEXT: the GEMM of the next panel left this panel's K range out, so that it
// could run beside this chain; each new s_a goes into the next panel's
// fields here instead, in FP32 (gx_out), from the block J[p][p+1]. Lane j
// owns next-panel spins 4 (32/RPW) u + 4 j + i, read as float4.
// The chain of panel p for the RPC = CW * RPW replica slots from slot0, on
// the CTA's first CW warps. Jb (and Jn when NEXT) hold the
// panel's blocks once `bar` completes its phase of parity `parity`; the caller
// issued their copies. With `pdl` the function orders itself after the
// stream's previous kernel (griddepcontrol) between the loads that kernel
// does not write and those it does. *s_ok is a shared word.
template <int RPW, bool NEXT, bool FP8, int CW = kChainWarps>
__device__ __forceinline__ void chain_body(const TcState& t, int p, const float* __restrict__ G,
                                           const float* __restrict__ gx_in, float* __restrict__ gx_out,
                                           bool g_early, bool pdl, int slot0, const float* Jb, const float* Jn,
                                           ChainSpin* cs_all, uint64_t* bar, uint32_t parity, int* s_ok)
{
    constexpr int LPR = 32 / RPW, SPL = kBM / LPR, RPC = CW * RPW;
    constexpr int kSplitCap = kChainMaxSplit / RPW;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int p0 = p * kBM;
    const int grp = lane / LPR, j = lane % LPR;
    const int r = warp * RPW + grp;
    const int slot = slot0 + r;
    // Programmatic launch: the kernel may start while the kernels it depends
    // on still run (each released its dependents only after its own
    // predecessors had completed). What those kernels do not write is read
    // first: this panel's old spins, the level state (the level step runs
    // between sweeps, before the sweep's first kernel) and, when `g_early`,
    // the fields, whose GEMM completed before the previous chain released
    // this one (the second panel of a pair). The previous chain's next-panel
    // fields (gx_in), and otherwise the fields, come after the wait.
    const bool valid = slot < t.R && t.active[slot];
    const float invT = valid ? t.invT[slot] : 0.f;  // idle groups compute and store nothing
    // RPC replicas x 32 four-spin pieces = RPW pieces per thread.
    static_assert(RPC * (kBM / 4) == RPW * CW * 32, "one piece per thread and replica slot");
    float4 part[RPW][kSplitCap], gx[RPW], so[RPW];
    uint2 sbw[RPW];  // the four spins' low-precision copies (BF16, or E4M3 in .x)
    auto load_fields = [&]() {
#pragma unroll
        for (int k = 0; k < RPW; ++k) {
            const int e = tid + k * CW * 32;
            const int rr = e / (kBM / 4), a4 = (e % (kBM / 4)) * 4;
            const int sl = slot0 + rr < t.R ? slot0 + rr : 0;
#pragma unroll
            for (int sp = 0; sp < kSplitCap; ++sp)
                part[k][sp] = sp < t.splitk
                                  ? *reinterpret_cast<const float4*>(G + ((size_t)sp * t.R_pad + sl) * kBM + a4)
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int e = tid + k * CW * 32;
        const int rr = e / (kBM / 4), a4 = (e % (kBM / 4)) * 4;
        const int sl = slot0 + rr < t.R ? slot0 + rr : 0;
        const size_t idx = (size_t)sl * t.n_pad + p0 + a4;
        so[k] = *reinterpret_cast<const float4*>(t.S + idx);
        if (FP8)
            sbw[k] = make_uint2(*reinterpret_cast<const uint32_t*>(t.S8 + idx), 0u);  // four E4M3
        else
            sbw[k] = *reinterpret_cast<const uint2*>(t.Sb + idx);  // four BF16
    }
    if (g_early) load_fields();
    if (pdl) {
        tc::pdl_wait();
        tc::pdl_launch_dependents();
    }
    if (!g_early) load_fields();
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int e = tid + k * CW * 32;
        const int rr = e / (kBM / 4), a4 = (e % (kBM / 4)) * 4;
        const int sl = slot0 + rr < t.R ? slot0 + rr : 0;
        gx[k] = gx_in ? *reinterpret_cast<const float4*>(gx_in + (size_t)sl * kBM + a4)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int e = tid + k * CW * 32;
        const int rr = e / (kBM / 4), a4 = (e % (kBM / 4)) * 4;
        float4 f = part[k][0];
#pragma unroll
        for (int sp = 1; sp < kSplitCap; ++sp) {
            if (sp < t.splitk) {
                f.x += part[k][sp].x;
                f.y += part[k][sp].y;
                f.z += part[k][sp].z;
                f.w += part[k][sp].w;
            }
        }
        if (gx_in) {
            f.x += gx[k].x;
            f.y += gx[k].y;
            f.z += gx[k].z;
            f.w += gx[k].w;
        }
        if (t.h) {
            const int a = p0 + a4;
            if (a + 0 < t.n) f.x += __ldg(t.h + a + 0);
            if (a + 1 < t.n) f.y += __ldg(t.h + a + 1);
            if (a + 2 < t.n) f.z += __ldg(t.h + a + 2);
            if (a + 3 < t.n) f.w += __ldg(t.h + a + 3);
        }
        float lo[4];
        if (FP8) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                __nv_fp8_e4m3 v;
                v.__x = (__nv_fp8_storage_t)((sbw[k].x >> (8 * i)) & 0xffu);
                lo[i] = float(v);
            }
        } else {
            lo[0] = __uint_as_float(sbw[k].x << 16);
            lo[1] = __uint_as_float(sbw[k].x & 0xffff0000u);
            lo[2] = __uint_as_float(sbw[k].y << 16);
            lo[3] = __uint_as_float(sbw[k].y & 0xffff0000u);
        }
        ChainSpin* d = cs_all + rr * kBM + a4;
        d[0] = ChainSpin{f.x, so[k].x, lo[0], 0.f};
        d[1] = ChainSpin{f.y, so[k].y, lo[1], 0.f};
        d[2] = ChainSpin{f.z, so[k].z, lo[2], 0.f};
        d[3] = ChainSpin{f.w, so[k].w, lo[3], 0.f};
    }
    if (tid == 0) *s_ok = tc::mbar_wait(bar, parity, t.counters + 2) ? 1 : 0;
    __syncthreads();
    if (!*s_ok) return;  // the error flag is set; the host reports it
    if (!__any_sync(0xffffffffu, valid)) return;  // the whole warp idle
    const ChainSpin* cs = cs_all + r * kBM;
    float g[SPL], sf[SPL], gn[NEXT ? SPL : 1];
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
        g[q] = cs[j + LPR * q].g;
        sf[q] = cs[j + LPR * q].s_old;
        if (NEXT) gn[q] = 0.f;
    }
    const int g0 = grp * LPR;  // the group's first lane
    // The step's argument in ex2 units, z_a = 2 log2(e) y_a with
    // y_a = (g_a + J[a-1][a] (s_{a-1} - sb_{a-1})) / T, is one FMA of the
    // previous step's new s: z_a = cz_a s_{a-1} + bz_a, where
    // cz_a = K J[a-1][a] / T and bz_a = K (g_a - J[a-1][a] sb_{a-1}) / T are
    // formed while the previous step's tanh is in flight.
    constexpr float kK = 2.8853900817779268f;     // 2 log2(e)
    constexpr float kKinv = 0.34657359027997264f;  // 1 / K
    constexpr float kSmallZ = 4e-3f * kK;          // |y| < 4e-3: tanh(y) = y to 2.2e-8
    const float kinv = kK * invT;
    ChainSpin c = cs[0];
    float cz = 0.f;  // J[-1][0] = 0
    float bz = kinv * __shfl_sync(0xffffffffu, g[0], g0);
    float snprev = 0.f, dloc = 0.f;
#pragma unroll
    for (int qa = 0; qa < SPL; ++qa) {
#pragma unroll 2
        for (int l = 0; l < LPR; ++l) {
            const int a = qa * LPR + l;
            const int an = a + 1 < kBM ? a + 1 : a;
            // What does not wait for this step's tanh: the broadcast of
            // g_{a+1} (before delta_a reaches it; its owner applies delta_a
            // below), the next step's operands and this step's J row.
            const float gsrc = l < LPR - 1 ? g[qa] : g[qa < SPL - 1 ? qa + 1 : SPL - 1];
            const float ghat_n = __shfl_sync(0xffffffffu, gsrc, g0 + (l + 1) % LPR);
            const ChainSpin c_n = cs[an];
            const float jp_n = Jb[a * kBM + an];  // J[a][a+1]
            const float* Jrow = Jb + a * kBM;
            float jr[SPL];
#pragma unroll
            for (int q = qa; q < SPL; ++q) jr[q] = Jrow[j + LPR * q];
            // The critical path: s_a = -tanh(y_a) = 2 / (1 + 2^z) - 1, SFU ex2
            // and rcp on the signed z (2^z overflows to +inf for z >> 0, giving
            // -1, and flushes to 0 for z << 0, giving +1); -y_a itself below
            // |y| = 4e-3.
            const float z = fmaf(cz, snprev, bz);
            float e, rc;
            asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(z));
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rc) : "f"(1.0f + e));
            const float big = fmaf(2.0f, rc, -1.0f);
            const float sn = fabsf(z) < kSmallZ ? -kKinv * z : big;
            const float delta = sn - c.s_old_bf;
            dloc = fmaxf(dloc, fabsf(sn - c.s_old));
            if (j == l) sf[qa] = sn;
#pragma unroll
            for (int q = qa; q < SPL; ++q) g[q] = fmaf(jr[q], delta, g[q]);
            if (NEXT) {
                const float4* Jnr = reinterpret_cast<const float4*>(Jn + a * kBM);
#pragma unroll
                for (int u = 0; u < SPL / 4; ++u) {
                    const float4 w = Jnr[LPR * u + j];
                    gn[4 * u + 0] = fmaf(w.x, sn, gn[4 * u + 0]);
                    gn[4 * u + 1] = fmaf(w.y, sn, gn[4 * u + 1]);
                    gn[4 * u + 2] = fmaf(w.z, sn, gn[4 * u + 2]);
                    gn[4 * u + 3] = fmaf(w.w, sn, gn[4 * u + 3]);
                }
            }
            cz = kinv * jp_n;
            bz = kinv * fmaf(-jp_n, c.s_old_bf, ghat_n);
            snprev = sn;
            c = c_n;
        }
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
        const int a = j + LPR * q;
        if (p0 + a < t.n) {
            const size_t idx = (size_t)slot * t.n_pad + p0 + a;
            t.S[idx] = sf[q];
            if (FP8)
                t.S8[idx] = __nv_fp8_e4m3(sf[q]).__x;
            else
                t.Sb[idx] = __float2bfloat16_rn(sf[q]);
        }
    }
    if (NEXT && gx_out) {  // the persistent sweeps' last panel has no next panel
#pragma unroll
        for (int u = 0; u < SPL / 4; ++u)
            *reinterpret_cast<float4*>(gx_out + (size_t)slot * kBM + 4 * (LPR * u + j)) =
                make_float4(gn[4 * u], gn[4 * u + 1], gn[4 * u + 2], gn[4 * u + 3]);
    }
    // every lane of the group computed every spin's change: dloc is the replica's maximum
    if (j == 0) t.d[slot] = fmaxf(t.d[slot], dloc);
}

// The chain as its own launch, one CTA per RPC replica slots. Thread 0 starts
// the copies of the panel's blocks (instance data, independent of the
// previous kernels) before chain_body's programmatic wait.
template <int RPW, bool NEXT, bool FP8, int CW>
__global__ void __launch_bounds__(CW * 32, 1)
    panel_chain_kernel(TcState t, int p, const float* __restrict__ G, const float* __restrict__ gx_in,
                       float* __restrict__ gx_out, int g_early)
{
    using L = ChainSmem<RPW, NEXT, CW>;
    extern __shared__ __align__(16) unsigned char chain_smem[];
    float* Jb = reinterpret_cast<float*>(chain_smem);  // J[p][p] (symmetric)
    float* Jn = Jb + kBM * kBM;                         // NEXT: J[p][p+1], row a = this panel's spin
    ChainSpin* cs_all = reinterpret_cast<ChainSpin*>(chain_smem + L::kBlocks * L::kJ);
    uint64_t* bar = reinterpret_cast<uint64_t*>(chain_smem + L::kBlocks * L::kJ + L::kCs);
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_barrier_init();
        tc::mbar_arrive_expect_tx(bar, L::kBlocks * L::kJ);
        tc::bulk_load(Jb, t.Jdiag + (size_t)p * kBM * kBM, L::kJ, bar);
        if (NEXT) tc::bulk_load(Jn, t.Jsup + (size_t)p * kBM * kBM, L::kJ, bar);
    }
    chain_body<RPW, NEXT, FP8, CW>(t, p, G, gx_in, gx_out, g_early != 0, true, blockIdx.x * (CW * RPW), Jb,
                                   Jn, cs_all, bar, 0u, &s_ok);
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
        if (t.S8)
            t.S8[idx] = __nv_fp8_e4m3(v).__x;
        else
            t.Sb[idx] = __float2bfloat16_rn(v);
    }
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < t.R; slot += gridDim.x * blockDim.x) {
        double T;
        const bool act = sched_first(t, (double)t.t0[t.rep[slot]], &T);
        t.T[slot] = T;
        t.invT[slot] = act ? sched_inv_t(T) : 0.f;
        t.active[slot] = act;
        t.levels[slot] = act ? 1 : 0;
        t.lvl_sweeps[slot] = 0;
        t.sweeps[slot] = 0;
        t.capped[slot] = 0;
        t.d[slot] = 0.f;
    }
}

// End of a sweep: the stopping rule and the level schedule per slot.
// The stopping rule and the level schedule of one active slot after a sweep.
__device__ __forceinline__ void advance_slot(const TcState& t, int slot)
{
    if (!t.active[slot]) return;
    const float dd = t.d[slot];
    t.d[slot] = 0.f;
    const int ls = t.lvl_sweeps[slot] + 1;
    t.sweeps[slot] += 1;
    double T = t.T[slot];
    const bool fixed = sched_fixed(t, T);
    const bool level_done = fixed ? ls >= t.fixed_sweeps : (dd <= t.d_min || ls >= t.k_max);
    if (level_done) {
        if (!fixed && !(dd <= t.d_min)) t.capped[slot] += 1;
        t.lvl_sweeps[slot] = 0;
        if (sched_advance(t, &T)) {
            t.T[slot] = T;
            t.levels[slot] += 1;
            t.invT[slot] = sched_inv_t(T);
        } else {
            t.active[slot] = 0;
        }
    } else {
        t.lvl_sweeps[slot] = ls;
    }
}

__global__ void tc_advance_kernel(TcState t)
{
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < t.R; slot += gridDim.x * blockDim.x)
        advance_slot(t, slot);
}

// ---------------------------------------------------------------------------
// Persistent sweeps for a partly active solve.
//
// Once fewer replicas are active than fill the GPU, a sweep is bound by its 64
// dependent panels (N = 8192) and, with one launch per GEMM and per chain, by
// the kernel boundaries between them. This kernel runs a whole batch of
// sweeps in one cooperative launch instead. Its first n_chain CTAs each own
// replica groups of kChainWarps * RPW slots and run their chains panel after
// panel; the other n_gemm CTAs run the panel GEMMs' (tile, split) items. The
// schedule is the overlap's: panel p's GEMM leaves panel p-1's K range out,
// so it needs the chains up to panel p-2 only, and chain p-1 supplies panel
// p-1's part of panel p's fields in FP32. The roles meet through two
// monotonic counters per panel of the batch (s = sweep * P + p):
//   gemm_done[s]  GEMM CTAs that finished their items of panel s (the chains
//                 of panel s wait for n_gemm);
//   chain_done[s] chain CTAs that finished panel s (panel s+2's GEMM waits
//                 for n_chain; a sweep's first panel, which leaves nothing
//                 out, waits for the previous sweep's last chain).
// Each role handles the panels in order, so every wait is for work that an
// earlier panel's waits did not depend on, and the cooperative launch keeps
// every CTA resident: the waits end. Each wait is bounded (a clock64 budget):
// on a timeout the CTA records the error, raises the shared abort word that
// every wait also watches, lets its copies in flight land and returns.
// ---------------------------------------------------------------------------
struct PersistSmem {
    static constexpr size_t kGemm = GemmSmem<128>::kBytes;
    template <int RPW>
    static constexpr size_t bytes()
    {
        return ChainSmem<RPW, true>::kBytes > kGemm ? (size_t)ChainSmem<RPW, true>::kBytes : kGemm;
    }
};

__device__ __forceinline__ int ld_acquire(const int32_t* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Thread 0 waits until *ctr >= target (acquire), giving up after the budget
// or when another CTA raised the abort word; the CTA learns the outcome.
__device__ bool wait_count(const int32_t* ctr, int32_t target, const TcPersist& pp, int32_t* err, int* s_flag)
{
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        int ok = 0;
        for (;;) {
            if (ld_acquire(ctr) >= target) { ok = 1; break; }
            if (*(volatile int32_t*)pp.abort) break;
            if (clock64() - t0 > pp.spin_budget) {
                atomicExch(err, tc::kErrTimeout);
                atomicExch(pp.abort, 1);
                break;
            }
            __nanosleep(40);
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Publishes this CTA's completion of a panel: its writes (made visible to
// the tensor maps' async proxy too) before the counter's increment.
__device__ __forceinline__ void publish(int32_t* ctr)
{
    fence_proxy_async_global();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1);
    }
}

template <int RPW, bool FP8>
__global__ void __launch_bounds__(kChainWarps * 32, 1)
    tc_sweeps_kernel(const __grid_constant__ CUtensorMap tmJ, const __grid_constant__ CUtensorMap tmS, TcState t,
                     TcPanel g, TcPersist pp)
{
    extern __shared__ __align__(1024) unsigned char psm[];
    __shared__ int s_flag;
    const int P = pp.P;
    int32_t* err = t.counters + 2;
    if (blockIdx.x < pp.n_chain) {
        // ---- chain role --------------------------------------------------
        using L = ChainSmem<RPW, true>;
        constexpr int RPC = kChainWarps * RPW;
        float* Jb = reinterpret_cast<float*>(psm);
        float* Jn = Jb + kBM * kBM;
        ChainSpin* cs_all = reinterpret_cast<ChainSpin*>(psm + L::kBlocks * L::kJ);
        uint64_t* bar = reinterpret_cast<uint64_t*>(psm + L::kBlocks * L::kJ + L::kCs);
        auto load_blocks = [&](int p) {
            tc::mbar_arrive_expect_tx(bar, L::kBlocks * L::kJ);
            tc::bulk_load(Jb, t.Jdiag + (size_t)p * kBM * kBM, L::kJ, bar);
            tc::bulk_load(Jn, t.Jsup + (size_t)p * kBM * kBM, L::kJ, bar);
        };
        if (threadIdx.x == 0) {
            tc::mbar_init(bar, 1);
            tc::fence_barrier_init();
            load_blocks(0);
        }
        __syncthreads();
        uint32_t loads = 1;  // block copies issued; the current one has parity (loads - 1) & 1
        bool failed = false;
        for (int w = 0; w < pp.sweeps && !failed; ++w) {
            for (int p = 0; p < P; ++p) {
                const int sidx = w * P + p;
                if (!wait_count(pp.gemm_done + sidx, pp.n_gemm, pp, err, &s_flag)) { failed = true; break; }
                for (int item = blockIdx.x; item < pp.chain_items; item += pp.n_chain) {
                    chain_body<RPW, true, FP8>(t, p, pp.G[sidx & 1], p > 0 ? pp.Gx[p & 1] : nullptr,
                                               p + 1 < P ? pp.Gx[(p + 1) & 1] : nullptr, true, false, item * RPC,
                                               Jb, Jn, cs_all, bar, (loads - 1) & 1u, &s_flag);
                    __syncthreads();
                    if (!s_flag) {
                        if (threadIdx.x == 0) atomicExch(pp.abort, 1);
                        failed = true;
                        break;
                    }
                }
                if (failed) break;
                if (p == P - 1) {
                    // the sweep's end for this CTA's slots: stopping rule and levels
                    for (int item = blockIdx.x; item < pp.chain_items; item += pp.n_chain)
                        for (int q = threadIdx.x; q < RPC; q += blockDim.x)
                            if (item * RPC + q < t.R) advance_slot(t, item * RPC + q);
                }
                __syncthreads();
                // the loops no longer read the blocks: copy the next panel's
                if (threadIdx.x == 0 && (w + 1 < pp.sweeps || p + 1 < P)) {
                    load_blocks(p + 1 < P ? p + 1 : 0);
                    ++loads;
                }
                publish(pp.chain_done + sidx);
            }
        }
        // a copy in flight lands before the CTA leaves
        if (threadIdx.x == 0) tc::mbar_wait(bar, (loads - 1) & 1u, err);
        __syncthreads();
        return;
    }
    // ---- GEMM role ---------------------------------------------------------
    using G = GemmSmem<128>;
    unsigned char* smem = (unsigned char*)(((uintptr_t)psm + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;
    unsigned char* sB = smem + kStages * G::kA;
    uint64_t* full = (uint64_t*)(sB + kStages * G::kB);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int q = 0; q < kStages; ++q) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        tc::tma_prefetch_desc(&tmJ);
        tc::tma_prefetch_desc(&tmS);
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, 128);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int kb_panel = g.fp8 ? 1 : 2;
    const int items = pp.gemm_tiles * pp.splitk;
    int it = 0, commits = 0;
    bool failed = false;
    for (int w = 0; w < pp.sweeps && !failed; ++w) {
        for (int p = 0; p < P; ++p) {
            const int sidx = w * P + p;
            // spins of every panel this GEMM reads: up to p-2 (panel p-1 is
            // left out), or up to the previous sweep's last panel for p = 0
            const int need = p == 0 ? sidx - 1 : sidx - 2;
            if (need >= 0 && !wait_count(pp.chain_done + need, pp.n_chain, pp, err, &s_flag)) {
                failed = true;
                break;
            }
            if (threadIdx.x == 0) fence_proxy_async_global();  // the chains' BF16 spins, for the TMA
            TcPanel gp = g;
            gp.p0 = p * kBM;
            gp.G = pp.G[sidx & 1];
            gp.skip_kb = p > 0 ? kb_panel * (p - 1) : -1;
            for (int item = blockIdx.x - pp.n_chain; item < items; item += pp.n_gemm) {
                bool committed = false;
                it = gemm_item<128, FP8>(&tmJ, &tmS, gp, (item / pp.splitk) * 128, item % pp.splitk, sA, sB, full,
                                         empty, done, tmem, it, commits, &committed);
                commits += committed ? 1 : 0;
                tc::tc_fence_before();
                __syncthreads();
                tc::tc_fence_after();
            }
            publish(pp.gemm_done + sidx);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
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

// The compaction's order of the slots below the prefix: active ones first,
// then finished ones, each in slot order (a block scan), and the new active
// prefix. One CTA of 1024 threads; thread k owns a contiguous run of slots.
__global__ void __launch_bounds__(1024) tc_compact_perm_kernel(TcState t, TcCompact cp, int prefix)
{
    __shared__ int s_warp[32];
    __shared__ int s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (prefix + 1023) / 1024;
    const int q0 = min(prefix, tid * per), q1 = min(prefix, q0 + per);
    int cnt = 0;
    for (int q = q0; q < q1; ++q) cnt += t.active[q] != 0;
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int v = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        s_warp[lane] = v;
        if (lane == 31) s_total = v;
    }
    __syncthreads();
    const int before = x - cnt + (warp > 0 ? s_warp[warp - 1] : 0);  // active slots before q0
    const int total = s_total;
    int a = before, f = total + (q0 - before);  // finished slots before q0 go after every active one
    for (int q = q0; q < q1; ++q) {
        if (t.active[q]) cp.perm[a++] = q;
        else cp.perm[f++] = q;
    }
    if (tid == 0) t.counters[0] = total;
}

// Gather every per-slot array of the slots below the prefix into the
// scratch in the new order.
__global__ void tc_compact_gather_kernel(TcState t, const int32_t* rep, TcCompact cp, int prefix)
{
    const size_t total = (size_t)prefix * t.n_pad;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(idx / t.n_pad), a = (int)(idx % t.n_pad);
        const size_t src = (size_t)cp.perm[q] * t.n_pad + a;
        cp.S[idx] = t.S[src];
        if (t.S8)
            cp.S8[idx] = t.S8[src];
        else
            cp.Sb[idx] = t.Sb[src];
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < prefix; q += gridDim.x * blockDim.x) {
        const int o = cp.perm[q];
        cp.T[q] = t.T[o];
        cp.invT[q] = t.invT[o];
        cp.d[q] = t.d[o];
        cp.active[q] = t.active[o];
        cp.levels[q] = t.levels[o];
        cp.lvl_sweeps[q] = t.lvl_sweeps[o];
        cp.sweeps[q] = t.sweeps[o];
        cp.capped[q] = t.capped[o];
        cp.rep[q] = rep[o];
    }
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
        t_last[t.rep[slot]] = t.levels[slot] > 0 ? t.T[slot] : 0.0;  // the last level's T (0: a quench)
}

}  // namespace

// Launch with programmatic stream serialization (programmatic dependent
// launch): the kernel may start while the stream's previous kernel still
// runs, and its griddepcontrol.wait orders it after that kernel. MARS_TC_PDL=0
// launches plainly.
cudaError_t launch_pdl(const void* k, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t st)
{
    static const bool on = [] {
        const char* v = std::getenv("MARS_TC_PDL");
        return !(v && *v && std::atoi(v) == 0);
    }();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = on ? 1 : 0;
    return cudaLaunchKernelExC(&cfg, k, args);
}

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
    const void* k = g.fp8 ? (bn == 64 ? (const void*)panel_gemm_kernel<64, true>
                                      : (const void*)panel_gemm_kernel<128, true>)
                          : (bn == 64 ? (const void*)panel_gemm_kernel<64, false>
                                      : (const void*)panel_gemm_kernel<128, false>);
    const size_t smem = tc_gemm_smem(bn);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    CUtensorMap a = tmJ, b = tmS;
    TcPanel c = g;
    void* args[] = {&a, &b, &c};
    return launch_pdl(k, dim3(n_tiles, splitk), dim3(128), args, smem, st);
}

cudaError_t launch_tc_pair_gemm(const CUtensorMap& tmJ, const CUtensorMap& tmS, const TcPanel& g, int n_tiles,
                                int splitk, cudaStream_t st)
{
    const void* k = g.fp8 ? (const void*)pair_gemm_kernel<128, true> : (const void*)pair_gemm_kernel<128, false>;
    const size_t smem = PairSmem<128>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (!g.G1 || g.skip_kb < 0) return cudaErrorInvalidValue;
    CUtensorMap a = tmJ, b = tmS;
    TcPanel c = g;
    void* args[] = {&a, &b, &c};
    return launch_pdl(k, dim3(n_tiles, splitk), dim3(128), args, smem, st);
}

template <int RPW, bool NEXT, bool FP8, int CW>
cudaError_t launch_chain_as(const TcState& t, int p, const float* G, const float* gx_in, float* gx_out,
                            int g_early, cudaStream_t st)
{
    constexpr int smem = ChainSmem<RPW, NEXT, CW>::kBytes;
    cudaError_t e = cudaFuncSetAttribute(panel_chain_kernel<RPW, NEXT, FP8, CW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int per_cta = CW * RPW;
    TcState tt = t;
    int pp = p;
    const float* a0 = G;
    const float* a1 = gx_in;
    float* a2 = gx_out;
    int ge = g_early;
    void* args[] = {&tt, &pp, &a0, &a1, &a2, &ge};
    return launch_pdl((const void*)panel_chain_kernel<RPW, NEXT, FP8, CW>, dim3((t.R + per_cta - 1) / per_cta),
                      dim3(CW * 32), args, smem, st);
}

template <bool FP8, int CW>
cudaError_t launch_chain_cw(const TcState& t, int p, int rpw, bool next, const float* G, const float* gx_in,
                            float* gx_out, int ge, cudaStream_t st)
{
    switch (rpw * 2 + (next ? 1 : 0)) {
    case 2: return launch_chain_as<1, false, FP8, CW>(t, p, G, gx_in, gx_out, ge, st);
    case 3: return launch_chain_as<1, true, FP8, CW>(t, p, G, gx_in, gx_out, ge, st);
    case 4: return launch_chain_as<2, false, FP8, CW>(t, p, G, gx_in, gx_out, ge, st);
    case 5: return launch_chain_as<2, true, FP8, CW>(t, p, G, gx_in, gx_out, ge, st);
    case 8: return launch_chain_as<4, false, FP8, CW>(t, p, G, gx_in, gx_out, ge, st);
    case 9: return launch_chain_as<4, true, FP8, CW>(t, p, G, gx_in, gx_out, ge, st);
    default: return cudaErrorInvalidValue;
    }
}

template <bool FP8>
cudaError_t launch_chain_lo(const TcState& t, int p, int rpw, int cw, bool next, const float* G,
                            const float* gx_in, float* gx_out, int ge, cudaStream_t st)
{
    return cw == 4 ? launch_chain_cw<FP8, 4>(t, p, rpw, next, G, gx_in, gx_out, ge, st)
                   : launch_chain_cw<FP8, kChainWarps>(t, p, rpw, next, G, gx_in, gx_out, ge, st);
}

cudaError_t launch_tc_chain(const TcState& t, int p, int rpw, int cw, const float* G, const float* gx_in,
                            float* gx_out, bool g_early, cudaStream_t st)
{
    if (rpw != 1 && rpw != 2 && rpw != 4) return cudaErrorInvalidValue;
    if (cw != 4 && cw != kChainWarps) return cudaErrorInvalidValue;
    if (t.splitk < 1 || t.splitk > kChainMaxSplit / rpw) return cudaErrorInvalidValue;
    // the CTA's slots must lie inside G's R_pad rows (R_pad is a multiple of 128)
    if (t.R_pad % (cw * rpw) != 0) return cudaErrorInvalidValue;
    const bool next = gx_out != nullptr;
    if (next && !t.Jsup) return cudaErrorInvalidValue;
    return t.S8 ? launch_chain_lo<true>(t, p, rpw, cw, next, G, gx_in, gx_out, g_early ? 1 : 0, st)
                : launch_chain_lo<false>(t, p, rpw, cw, next, G, gx_in, gx_out, g_early ? 1 : 0, st);
}

cudaError_t launch_tc_init(const TcState& t, cudaStream_t st)
{
    tc_init_kernel<<<1024, 256, 0, st>>>(t);
    return cudaGetLastError();
}

size_t tc_sweeps_smem(int rpw)
{
    return rpw == 1 ? PersistSmem::bytes<1>() : rpw == 2 ? PersistSmem::bytes<2>() : PersistSmem::bytes<4>();
}

template <int RPW, bool FP8>
cudaError_t launch_sweeps_as(const CUtensorMap& tmJ, const CUtensorMap& tmS, const TcState& t, const TcPanel& g,
                             const TcPersist& pp, cudaStream_t st)
{
    const void* k = (const void*)tc_sweeps_kernel<RPW, FP8>;
    const size_t smem = PersistSmem::bytes<RPW>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    CUtensorMap a = tmJ, b = tmS;
    TcState c = t;
    TcPanel d = g;
    TcPersist q = pp;
    void* args[] = {&a, &b, &c, &d, &q};
    return cudaLaunchCooperativeKernel(k, dim3(pp.n_chain + pp.n_gemm), dim3(kChainWarps * 32), args, smem, st);
}

cudaError_t launch_tc_sweeps(const CUtensorMap& tmJ, const CUtensorMap& tmS, const TcState& t, const TcPanel& g,
                             const TcPersist& pp, int rpw, cudaStream_t st)
{
    if (pp.n_chain < 1 || pp.n_gemm < 1 || pp.sweeps < 1 || pp.splitk < 1 || pp.splitk > kChainMaxSplit / rpw)
        return cudaErrorInvalidValue;
    const bool fp8 = g.fp8 != 0;
    switch (rpw) {
    case 1: return fp8 ? launch_sweeps_as<1, true>(tmJ, tmS, t, g, pp, st) : launch_sweeps_as<1, false>(tmJ, tmS, t, g, pp, st);
    case 2: return fp8 ? launch_sweeps_as<2, true>(tmJ, tmS, t, g, pp, st) : launch_sweeps_as<2, false>(tmJ, tmS, t, g, pp, st);
    case 4: return fp8 ? launch_sweeps_as<4, true>(tmJ, tmS, t, g, pp, st) : launch_sweeps_as<4, false>(tmJ, tmS, t, g, pp, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tc_advance(const TcState& t, cudaStream_t st)
{
    tc_advance_kernel<<<(t.R + 255) / 256, 256, 0, st>>>(t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tc_prefix_kernel<<<1, 1024, 0, st>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_tc_compact(const TcState& t, int32_t* rep, const TcCompact& cp, int prefix, cudaStream_t st)
{
    if (prefix <= 0 || prefix > t.R) return cudaErrorInvalidValue;
    tc_compact_perm_kernel<<<1, 1024, 0, st>>>(t, cp, prefix);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tc_compact_gather_kernel<<<1024, 256, 0, st>>>(t, rep, cp, prefix);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t rows = (size_t)prefix * t.n_pad;
    auto back = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st);
    };
    if ((e = back(t.S, cp.S, rows * sizeof(float))) != cudaSuccess) return e;
    if (t.S8) {
        if ((e = back(t.S8, cp.S8, rows)) != cudaSuccess) return e;
    } else if ((e = back(t.Sb, cp.Sb, rows * sizeof(__nv_bfloat16))) != cudaSuccess) {
        return e;
    }
    const size_t q = (size_t)prefix;
    if ((e = back(t.T, cp.T, q * sizeof(double))) != cudaSuccess) return e;
    if ((e = back(t.invT, cp.invT, q * sizeof(float))) != cudaSuccess) return e;
    if ((e = back(t.d, cp.d, q * sizeof(float))) != cudaSuccess) return e;
    if ((e = back(t.active, cp.active, q * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = back(t.levels, cp.levels, q * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = back(t.lvl_sweeps, cp.lvl_sweeps, q * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = back(t.sweeps, cp.sweeps, q * sizeof(int32_t))) != cudaSuccess) return e;
    if ((e = back(t.capped, cp.capped, q * sizeof(int32_t))) != cudaSuccess) return e;
    return back(rep, cp.rep, q * sizeof(int32_t));
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
