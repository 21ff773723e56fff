"""Noisy mean-field annealing (Section 2's NMFA) on the GPU against the FP64
oracle, through the C ABI.

NMFA is the alternative epilogue the library runs on the same local-field
engines: the synchronous dense FP32 kernels and the CSR walk. Every
iteration normalises each spin's field by sqrt(h_i^2 + sum_j J_ij^2), adds
counter-based Gaussian noise, takes -tanh(. / T) and mixes it into the old
value with weight alpha; one iteration per temperature level. The bar is the
strict trajectory tier: per-replica m within 1e-5 max-abs of the oracle (the
GPU's FP32 noise differs from the oracle's FP64 Box-Muller by a few FP32
ulps; the normalised, mixed update is well conditioned: the oracle's own
change under a one-ulp change of m0 or of sigma is about 1e-7 on these
instances).
"""
import numpy as np
import pytest

import oracle as O
from paper_1907_05124_gb300 import instances as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def _cases():
    rng = np.random.default_rng(5)
    h = rng.normal(size=150)
    return {
        "sk_pm1": (O.Instance.dense(I.sk_pm1(96, 1)), "dense", I.sk_pm1(96, 1), None),
        "sk_gauss_field": (O.Instance.dense(I.sk_gauss(150, 2), h), "dense", I.sk_gauss(150, 2), h),
        "lattice": (O.Instance.csr(I.ea_lattice(20, 2, 3)), "csr", I.ea_lattice(20, 2, 3), None),
        "er_one": (O.Instance.csr(I.er_graph(700, 8, 4, "one")), "csr", I.er_graph(700, 8, 4, "one"), None),
    }


@pytest.mark.parametrize("sigma", [0.0, 0.3])
@pytest.mark.parametrize("name", ["sk_pm1", "sk_gauss_field", "lattice", "er_one"])
def test_nmfa_trajectories_match_oracle(ctx, name, sigma):
    oi, kind, data, h = _cases()[name]
    inst = ctx.add_dense(data, h=h) if kind == "dense" else ctx.add_csr(*data, h=h)
    R = 48
    m0, t0 = I.replica_inputs(R, oi.n, 1.5, 4.9, 7)
    t0 = (np.floor(t0) + 0.5 + 0.5 * (t0 - np.floor(t0))).astype(np.float32)  # every level at T >= 0.5
    kw = dict(c_step=1.0, alpha=0.35, sigma=sigma, seed=21, stream=2)
    g = ctx.solve(inst, R, float(t0.min()), float(t0.max()), m0=m0, t0=t0, method="nmfa",
                  outputs=("m_final", "energies", "spins", "sweeps", "levels"), **kw)
    o = O.nmfa_solve(oi, m0, t0, nthreads=8, **kw)
    err = float(np.abs(g.m_final - o["m"]).max())
    assert err <= TOL, err
    assert np.array_equal(g.replica_levels, o["levels"])
    assert np.array_equal(g.replica_sweeps, o["levels"])  # one iteration per level
    assert np.array_equal(g.energies, O.energies(oi, g.spins))
    if sigma > 0:  # the noise moved the trajectory
        z = O.nmfa_solve(oi, m0, t0, nthreads=8, **dict(kw, sigma=0.0))
        assert np.abs(z["m"] - o["m"]).max() > 1e-2
    ctx.free(inst)


def test_nmfa_drawn_start_states_and_replica_streams(ctx):
    """Start states and temperatures drawn on the device (the oracle draws
    the same ones), noise keyed by (seed, stream, replica, iteration, spin)."""
    csr = I.ea_lattice(16, 2, 8)
    inst = ctx.add_csr(*csr)
    oi = O.Instance.csr(csr)
    R, tmin, tmax = 40, 2.0, 5.0
    g = ctx.solve(inst, R, tmin, tmax, seed=9, stream=3, method="nmfa", alpha=0.6, sigma=0.2,
                  outputs=("m_final",))
    m0, t0 = O.draw_replicas(9, R, csr.n, tmin, tmax, stream=3)
    o = O.nmfa_solve(oi, m0, t0, c_step=1.0, alpha=0.6, sigma=0.2, seed=9, stream=3)
    # the oracle's own change under a one-ulp change of m0 is below 1e-6 here
    assert float(np.abs(g.m_final - o["m"]).max()) <= TOL
    ctx.free(inst)


def test_nmfa_served_equals_blocking(ctx):
    import time
    inst = ctx.add_csr(*I.er_graph(900, 10, 6, "pm1"))
    kw = dict(seed=4, method="nmfa", alpha=0.5, sigma=0.25)
    req = ctx.submit(inst, 64, 0.0, 6.0, **kw)
    t = time.time()
    res = None
    while res is None:
        res = ctx.poll(req)
        assert time.time() - t < 60
        time.sleep(0.001)
    ref = ctx.solve(inst, 64, 0.0, 6.0, **kw)
    assert res.best_energy == ref.best_energy and res.best_replica == ref.best_replica
    assert res.sweeps == ref.sweeps
    assert np.array_equal(res.best_spins, ref.best_spins)
    ctx.free(inst)


def test_nmfa_rejections(ctx):
    from paper_1907_05124_gb300.mars import MarsError
    d = ctx.add_dense(I.sk_pm1(64, 0))
    for kw in (dict(precision="bf16"), dict(quench=True), dict(alpha=1.5), dict(sigma=-1.0)):
        with pytest.raises(MarsError):
            ctx.solve(d, 8, 0.0, 4.0, method="nmfa", **kw)
    ctx.free(d)
