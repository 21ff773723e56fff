"""Sparse descent with the magnetisations in global memory (n too large for
even one replica's m in shared memory), against the FP64 oracle. Two kernels
run it: the level-synchronous one (the default: every replica resident, one
grid-wide launch per level of the schedule) and the per-CTA slabs (each CTA
drains the replica queue on its own slab, MARS_SELL_WIDE=0).

- Fixed-sweep trajectories of Algorithm 1 (Section 3), strict tier (one sweep
  per level, at most three levels, every level at T >= C_step / 2 = 1,
  max-abs 1e-5 in m), exact sweep and level counts, and exact energies of the
  returned spins, for both kernels:
  - 3-D +-J lattice L = 40 (n = 64000, degree 6: the unrolled +-1-word
    kernels) with R = 320 replicas, so the per-CTA kernel refills slots from
    the replica queue;
  - Erdos-Renyi graph, n = 60000, mean degree 5, Gaussian weights (general
    (column, weight) couplings), R = 5.
- Under the paper's stopping rule the two kernels return identical outputs
  (spins, final magnetisations, energies, sweep, level and capped-level
  counts), since each spin's field is summed in the same order and passes
  through the same tanh: slot widths 1, 2 and 4, partly filled groups,
  replicas that visit no level, a field h, and the geometric schedule with a
  quench level.
- The 3-D lattice with N = 10^6 and R = 608 (the HBM workload's own size):
  strict-tier trajectories of sampled replicas against the oracle, and a
  whole solve under the stopping rule whose energies are the exact energies
  of the returned spins.
"""
import numpy as np
import pytest

import oracle as O
from paper_1907_05124_gb300 import instances as I

from test_gpu_parity import STRICT_LEVELS, check_trajectory, floored_t0

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05124_gb300 import build, mars
    build.build()
    c = mars.Context(0)
    yield c
    c.close()


def gaussian_weights(csr, seed):
    """The same graph with N(0, 1) weights, one per undirected edge."""
    n = csr.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(csr.row_ptr))
    cols = csr.col.astype(np.int64)
    key = np.minimum(rows, cols) * n + np.maximum(rows, cols)
    uniq = np.unique(key)
    w = np.random.default_rng(seed).normal(size=uniq.size)
    return I.Csr(csr.row_ptr, csr.col, w[np.searchsorted(uniq, key)])


@pytest.fixture(params=["wide", "per_cta"])
def kernel(request, monkeypatch):
    monkeypatch.setenv("MARS_SELL_WIDE", "1" if request.param == "wide" else "0")
    return request.param


@pytest.mark.parametrize("case", ["ea3d_40_pm1", "er_60000_gauss"])
def test_slab_fixed_sweep_trajectories(ctx, case, kernel):
    if case == "ea3d_40_pm1":
        csr, R = I.ea_lattice(40, 3, 6), 320
    else:
        csr, R = gaussian_weights(I.er_graph(60000, 5, 12, "pm1"), 13), 5
    tmax, c = 8.0, 2.0
    order = I.greedy_colour_order(csr)
    inst = ctx.add_csr(*csr, order=order)
    m0, t0 = I.replica_inputs(R, csr.n, 0.0, tmax, 41)
    t0 = floored_t0(t0, c, max_levels=STRICT_LEVELS)
    g = ctx.solve(inst, R, 0.0, tmax, c_step=c, fixed_sweeps=1, m0=m0, t0=t0,
                  outputs=("m_final", "sweeps", "levels", "energies", "spins"))
    oi = O.Instance.csr(csr)
    o = O.mars_solve(oi, m0, t0, c_step=c, fixed_sweeps=1, order=order)
    check_trajectory(g.m_final, o["m"], "strict")
    assert np.array_equal(g.replica_sweeps, o["sweeps"])
    assert np.array_equal(g.replica_levels, o["levels"])
    assert np.array_equal(g.energies, O.energies(oi, g.spins))
    ctx.free(inst)


def _solve_both(ctx, monkeypatch, inst, R, **kw):
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("MARS_SELL_WIDE", mode)
        out[mode] = ctx.solve(inst, R, outputs=("m_final", "sweeps", "levels", "capped", "energies", "spins"),
                              **kw)
    return out["1"], out["0"]


def _same(a, b):
    assert a.best_energy == b.best_energy and a.best_replica == b.best_replica
    assert np.array_equal(a.energies, b.energies)
    assert np.array_equal(a.spins, b.spins)
    assert np.array_equal(a.m_final, b.m_final)
    assert np.array_equal(a.replica_sweeps, b.replica_sweeps)
    assert np.array_equal(a.replica_levels, b.replica_levels)
    assert np.array_equal(a.replica_capped, b.replica_capped)


@pytest.mark.parametrize("rt", [1, 2, 4])
def test_level_synchronous_equals_per_cta_kernel(ctx, monkeypatch, rt):
    """The paper's stopping rule (d_min = 1e-4, k_max = 1000) on the L = 40
    lattice; R = 37 leaves the last group partly filled, and replicas with
    T0 < C_step visit no level (their spins are sign(m0))."""
    csr = I.ea_lattice(40, 3, 6)
    inst = ctx.add_csr(*csr, order=I.greedy_colour_order(csr))
    ctx.set_shape(inst, sell_rt=rt)
    R, tmax = 37, 5.0
    m0, t0 = I.replica_inputs(R, csr.n, 0.0, tmax, 51)
    t0[:3] = [0.2, 0.5, 0.9]
    a, b = _solve_both(ctx, monkeypatch, inst, R, t_min=0.0, t_max=tmax, c_step=1.0, m0=m0, t0=t0)
    _same(a, b)
    assert (a.replica_levels[:3] == 0).all()
    assert a.replica_levels.max() >= 4 and a.replica_sweeps.max() > a.replica_levels.max()
    assert a.level_launches > 0 and b.level_launches == 0
    ctx.free(inst)


def test_level_synchronous_equals_per_cta_field_and_quench(ctx, monkeypatch):
    """General (column, weight) couplings with a field h (the update adds h_i
    to the field), and the geometric schedule ending in a quench level."""
    csr = gaussian_weights(I.er_graph(60000, 5, 14, "pm1"), 15)
    h = np.random.default_rng(16).normal(scale=0.3, size=csr.n)
    inst = ctx.add_csr(*csr, h=h, order=I.greedy_colour_order(csr))
    ctx.set_shape(inst, sell_rt=4)
    R = 10
    m0, t0 = I.replica_inputs(R, csr.n, 0.5, 3.0, 17)
    a, b = _solve_both(ctx, monkeypatch, inst, R, t_min=0.5, t_max=3.0, m0=m0, t0=t0,
                       geometric=0.6, t_floor=0.3, quench=True)
    _same(a, b)
    ctx.free(inst)


def test_full_size_lattice_level_synchronous(ctx, monkeypatch):
    """N = 10^6 (3-D L = 100), R = 608, the HBM workload's size: one sweep per
    level, strict tier, on 6 sampled replicas (the oracle sweeps a replica
    in well under a second); then the paper's stopping rule on the same
    instance, with exact energies of sampled returned spins."""
    monkeypatch.setenv("MARS_SELL_WIDE", "1")
    csr = I.ea_lattice(100, 3, 0)
    order = I.greedy_colour_order(csr)
    inst = ctx.add_csr(*csr, order=order)
    R, tmax, c = 608, 6.0, 2.0
    m0, t0 = I.replica_inputs(R, csr.n, 0.0, tmax, 61)
    t0 = floored_t0(t0, c, max_levels=STRICT_LEVELS)
    g = ctx.solve(inst, R, 0.0, tmax, c_step=c, fixed_sweeps=1, m0=m0, t0=t0,
                  outputs=("m_final", "sweeps", "levels"))
    idx = np.unique(np.concatenate([[0, R - 1], np.random.default_rng(62).choice(R, 4, replace=False)]))
    oi = O.Instance.csr(csr)
    o = O.mars_solve(oi, m0[idx], t0[idx], c_step=c, fixed_sweeps=1, order=order, nthreads=len(idx))
    check_trajectory(g.m_final[idx], o["m"], "strict")
    assert np.array_equal(g.replica_sweeps[idx], o["sweeps"])
    assert np.array_equal(g.replica_levels[idx], o["levels"])
    r = ctx.solve(inst, R, 0.0, tmax, c_step=1.0, seed=3, outputs=("energies", "spins", "levels", "sweeps"))
    pick = np.unique(np.concatenate([[r.best_replica], idx]))
    assert np.array_equal(r.energies[pick], O.energies(oi, r.spins[pick]))
    assert r.best_energy == r.energies.min()
    assert (r.replica_sweeps >= r.replica_levels).all()
    assert r.level_launches > 0 and r.level_seconds > 0
    ctx.free(inst)


@pytest.mark.parametrize("rt", [1, 4])
def test_staged_and_register_level_kernels_agree(ctx, monkeypatch, rt):
    """On a regular lattice the level launch stages the next slice's neighbour
    rows in shared memory by asynchronous copies; MARS_WIDE_STAGED=0 keeps
    them in registers. Both sum each field in the same order: identical
    outputs under the paper's stopping rule."""
    monkeypatch.setenv("MARS_SELL_WIDE", "1")
    csr = I.ea_lattice(40, 3, 8)
    inst = ctx.add_csr(*csr, order=I.greedy_colour_order(csr))
    ctx.set_shape(inst, sell_rt=rt)
    R = 21
    m0, t0 = I.replica_inputs(R, csr.n, 0.0, 5.0, 81)
    out = {}
    for staged in ("1", "0"):
        monkeypatch.setenv("MARS_WIDE_STAGED", staged)
        out[staged] = ctx.solve(inst, R, 0.0, 5.0, m0=m0, t0=t0,
                                outputs=("m_final", "sweeps", "levels", "capped", "energies", "spins"))
    _same(out["1"], out["0"])
    ctx.free(inst)
