"""Sparse descent with the magnetisations in global-memory slabs (n too large
for even one replica's m in shared memory), against the FP64 oracle:
fixed-sweep trajectories of Algorithm 1 (Section 3), strict tier (one sweep
per level, at most three levels, every level at T >= C_step / 2 = 1, max-abs
1e-5 in m), exact sweep and level counts, and exact energies of the returned
spins.

- 3-D +-J lattice L = 40 (n = 64000, degree 6: the unrolled +-1-word kernel)
  with R = 320 replicas, more than one slot pair per SM holds, so slots are
  refilled from the replica queue;
- Erdos-Renyi graph, n = 60000, mean degree 5, Gaussian weights (general
  (column, weight) couplings), R = 5.
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


@pytest.mark.parametrize("case", ["ea3d_40_pm1", "er_60000_gauss"])
def test_slab_fixed_sweep_trajectories(ctx, case):
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
