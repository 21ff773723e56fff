// Temperature schedule of a descent.
//
// Section 3, Algorithm 1: before each level T <- T - C_step, and levels run
// while T > 0. Two labelled variants (not the paper's schedule): geometric
// cooling, T <- r T while T > t_floor; and a final quench level that takes
// Algorithm 1's last decrement to the T -> 0+ limit of the update,
// s_i <- -sgn(Phi_i). The quench level is marked by T == 0 (every other level
// has T > 0) and runs at 1/T = kQuenchInvT: a nonzero FP32 field then gives
// |Phi / T| >= 1e20 or so, whose tanh is exactly +-1 in every tanh the kernels
// use, and a zero field gives 0, so the update needs no branch. The quench
// level keeps the stopping rule (d <= d_min or k_max sweeps) even when the
// other levels run a fixed number of sweeps.
#pragma once

namespace mars {

constexpr float kQuenchInvT = 1e30f;

template <class S>
__host__ __device__ inline double sched_next(const S& s, double T)
{
    return s.geometric ? T * s.cool_ratio : T - s.c_step;
}

template <class S>
__host__ __device__ inline bool sched_runs(const S& s, double T)
{
    return T > (s.geometric ? s.t_floor : 0.0);
}

// The first level's temperature from the start temperature t0; false when the
// replica visits no level (then its result is sign(m0)).
template <class S>
__host__ __device__ inline bool sched_first(const S& s, double t0, double* T)
{
    const double Tn = sched_next(s, t0);
    if (sched_runs(s, Tn)) {
        *T = Tn;
        return true;
    }
    *T = 0.0;
    return s.quench != 0;
}

// After the level at *T ended: the next level's temperature; false when the
// descent is over.
template <class S>
__host__ __device__ inline bool sched_advance(const S& s, double* T)
{
    if (*T == 0.0) return false;  // the quench level is the last
    const double Tn = sched_next(s, *T);
    if (sched_runs(s, Tn)) {
        *T = Tn;
        return true;
    }
    *T = 0.0;
    return s.quench != 0;
}

__host__ __device__ inline float sched_inv_t(double T) { return T > 0.0 ? (float)(1.0 / T) : kQuenchInvT; }

// Whether the level at T runs a fixed number of sweeps.
template <class S>
__host__ __device__ inline bool sched_fixed(const S& s, double T)
{
    return s.fixed_sweeps > 0 && T != 0.0;
}

}  // namespace mars
