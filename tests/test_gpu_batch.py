"""mars_solve_batch: several instances in one persistent launch.

Each replica's arithmetic does not depend on which CTA, slot width or coupling
format runs it, so every job of a batch must return exactly what a separate
mars_solve returns for the same instance and parameters.
"""
import numpy as np
import pytest

import oracle as O
from paper_1907_05124_gb300 import instances as I

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


def _same(a, b):
    assert a.best_energy == b.best_energy
    assert a.best_replica == b.best_replica
    assert a.hits == b.hits
    assert a.sweeps == b.sweeps and a.levels == b.levels and a.capped_levels == b.capped_levels
    assert a.mean_energy == pytest.approx(b.mean_energy, rel=1e-12)
    assert np.array_equal(a.best_spins, b.best_spins)


def test_batch_equals_separate_solves(ctx):
    graphs = [I.er_graph(500, 6, 1, "pm1"), I.er_graph(1200, 12, 2, "one"),
              I.ea_lattice(30, 2, 3), I.ea_lattice(8, 3, 4), I.er_graph(3000, 20, 5, "pm1")]
    t_max = [5.0, 12.0, 4.0, 5.0, 9.0]
    Rs = [300, 64, 257, 33, 128]
    insts = [ctx.add_csr(*g) for g in graphs]
    jobs = [(inst, R, 0.0, tm, {"seed": 7 + j}) for j, (inst, R, tm) in enumerate(zip(insts, Rs, t_max))]
    batch = ctx.solve_batch(jobs)
    for (inst, R, lo, hi, kw), b, g in zip(jobs, batch, graphs):
        ref = ctx.solve(inst, R, lo, hi, seed=kw["seed"], outputs=("energies",))
        _same(b, ref)
        assert b.best_energy == O.energy(O.Instance.csr(g), b.best_spins)
    for inst in insts:
        ctx.free(inst)


def test_batch_fixed_sweeps_with_start_states_matches_oracle(ctx):
    g1, g2 = I.er_graph(400, 7, 8, "pm1"), I.ea_lattice(12, 2, 9)
    i1, i2 = ctx.add_csr(*g1), ctx.add_csr(*g2)
    m1, t1 = I.replica_inputs(9, g1.n, 0.0, 3.9, 10)
    m2, t2 = I.replica_inputs(5, g2.n, 0.0, 3.9, 11)
    out = ctx.solve_batch([(i1, 9, 0.0, 3.9, {"m0": m1, "t0": t1, "fixed_sweeps": 1}),
                           (i2, 5, 0.0, 3.9, {"m0": m2, "t0": t2, "fixed_sweeps": 1})])
    for res, g, m0, t0 in ((out[0], g1, m1, t1), (out[1], g2, m2, t2)):
        o = O.mars_solve(O.Instance.csr(g), m0, t0, fixed_sweeps=1, order=None, want_m=False)
        # the library's colour order differs from 0..n-1, so compare what is
        # order-free: the energy of the returned spins and the sweep counts
        assert res.sweeps == int(o["sweeps"].sum())
        assert res.best_energy == O.energy(O.Instance.csr(g), res.best_spins)
    ctx.free(i1)
    ctx.free(i2)


def test_batch_float_weights_exact_energies(ctx):
    g = I.er_graph(900, 9, 12, "pm1")
    g = I.Csr(g.row_ptr, g.col, g.val * 0.37)
    h = np.random.default_rng(1).normal(size=900) * 0.2
    inst = ctx.add_csr(*g, h=h)
    lat = ctx.add_csr(*I.ea_lattice(20, 2, 13))
    out = ctx.solve_batch([(inst, 64, 0.0, 3.0, {"seed": 1}), (lat, 64, 0.0, 4.0, {"seed": 2})])
    assert out[0].best_energy == O.energy(O.Instance.csr(g, h), out[0].best_spins)
    assert out[0].energy_err_bound == 0.0
    ref = ctx.solve(inst, 64, 0.0, 3.0, seed=1)
    _same(out[0], ref)
    ctx.free(inst)
    ctx.free(lat)


def test_batch_rejects_dense_and_bad_jobs(ctx):
    from paper_1907_05124_gb300.mars import MarsError
    d = ctx.add_dense(I.sk_pm1(32, 0))
    s = ctx.add_csr(*I.ea_lattice(6, 2, 0))
    with pytest.raises(MarsError):
        ctx.solve_batch([(s, 8, 0.0, 4.0, {}), (d, 8, 0.0, 4.0, {})])
    with pytest.raises(MarsError):
        ctx.solve_batch([(s, 0, 0.0, 4.0, {})])
    ctx.free(d)
    ctx.free(s)


def test_batch_mixes_slot_widths(ctx):
    """A 3-D L=32 lattice (N = 32768: one replica slot per CTA fits on chip)
    shares the launch with small graphs that run two slots per CTA; every job
    returns exactly what a separate mars_solve returns."""
    graphs = [I.ea_lattice(32, 3, 21), I.er_graph(900, 6, 22, "pm1"), I.ea_lattice(24, 2, 23)]
    insts = [ctx.add_csr(*g) for g in graphs]
    Rs, tmax = [48, 200, 130], [6.0, 6.0, 4.0]
    jobs = [(i, R, 0.0, tm, {"seed": 60 + j}) for j, (i, R, tm) in enumerate(zip(insts, Rs, tmax))]
    out = ctx.solve_batch(jobs)
    for (inst, R, lo, hi, kw), b in zip(jobs, out):
        _same(b, ctx.solve(inst, R, lo, hi, seed=kw["seed"], outputs=("energies",)))
    for inst in insts:
        ctx.free(inst)


def test_batch_with_schedule_variants(ctx):
    """Geometric cooling and the quench level travel with each job."""
    g1, g2 = I.er_graph(600, 6, 27, "pm1"), I.ea_lattice(16, 2, 28)
    i1, i2 = ctx.add_csr(*g1), ctx.add_csr(*g2)
    kw1 = {"seed": 3, "geometric": 0.8, "t_floor": 0.3, "quench": True}
    kw2 = {"seed": 4, "quench": True}
    out = ctx.solve_batch([(i1, 80, 0.0, 6.0, kw1), (i2, 60, 0.0, 4.0, kw2)])
    _same(out[0], ctx.solve(i1, 80, 0.0, 6.0, seed=3, geometric=0.8, t_floor=0.3, quench=True))
    _same(out[1], ctx.solve(i2, 60, 0.0, 4.0, seed=4, quench=True))
    ctx.free(i1)
    ctx.free(i2)
