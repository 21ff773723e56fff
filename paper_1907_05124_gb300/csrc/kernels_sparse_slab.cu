// Sparse MARS descent (Section 3, Algorithm 1) for instances whose
// magnetisations do not fit in shared memory even for one replica: the
// sliced-ELL job of sell_job.cuh with each CTA's m[i*RT + k] in its own slab
// of global memory.
//
// A sweep streams the slab level by level. The lanes of a warp own the 32
// consecutive rows of a slice, so their stores, and on lattices their
// RT-wide neighbour gathers (consecutive labels), are coalesced; the
// couplings come through L1 and L2 and serve all RT replicas of the CTA. The
// slab is written by the kernel, so it is read with plain coherent loads,
// never through the read-only path; a block barrier after each level makes
// the level's stores visible to the whole CTA. One 1024-thread CTA per SM.
#include "sell_job.cuh"

namespace mars {
namespace {

template <int RT, int FMT, int DEG>
__global__ void __launch_bounds__(1024, 1) sparse_slab_kernel(DevInstance in, DevSolve s)
{
    __shared__ SlotState<RT, 32> S;
    float* m = s.m_scratch + (size_t)blockIdx.x * sell_slab_floats(in.n, RT);
    run_job<RT, 1024, FMT, DEG>(in, s, m, S);
}

// +-1 words (format 1), unrolled for the lattices' degrees 4 and 6; general
// (column, weight) pairs (format 0) with the degree read per slice.
template <int RT>
const void* pick_rt(int fmt, int deg)
{
    if (fmt == 0) return (const void*)sparse_slab_kernel<RT, 0, 0>;
    return deg == 4 ? (const void*)sparse_slab_kernel<RT, 1, 4>
         : deg == 6 ? (const void*)sparse_slab_kernel<RT, 1, 6>
                    : (const void*)sparse_slab_kernel<RT, 1, 0>;
}

}  // namespace

const void* pick_sell_slab(int rt, int fmt, int deg)
{
    if (fmt != 0 && fmt != 1) return nullptr;
    switch (rt) {
    case 1: return pick_rt<1>(fmt, deg);
    case 2: return pick_rt<2>(fmt, deg);
    case 4: return pick_rt<4>(fmt, deg);
    }
    return nullptr;
}

}  // namespace mars
