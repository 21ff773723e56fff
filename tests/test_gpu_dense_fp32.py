"""Dense FP32 descent at the sizes that pick each of its kernels.

Fixed-sweep trajectories (Algorithm 1, Section 3) against the FP64 oracle,
strict tier (one sweep per level, at most three levels, every level at
T >= c_step / 2), max-abs 1e-5 in m:

- n = 4, 8: the ring of row buffers holds the whole matrix (n = 4: each
  stage always holds the same row) and the rows wrap every sweep;
- n = 8000, 9000: three and two row buffers;
- n = 12000: no room for two row buffers beside the replicas' m, so every
  warp reads J through the read-only cache (float4 rows);
- n = 14402: m no longer fits in shared memory (global scratch rows) and
  n % 4 != 0 (scalar rows).

R = 5 leaves the second CTA with one live replica and three warps that only
take part in the row pipeline.
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


@pytest.mark.parametrize("n", [4, 8])
def test_tiny_n_row_ring_wraps(ctx, n):
    J = I.sk_pm1(n, 5)
    inst = ctx.add_dense(J)
    R, tmax = 5, 4.0
    m0, t0 = I.replica_inputs(R, n, 0.0, tmax, 29)
    t0 = floored_t0(t0, 1.0, max_levels=STRICT_LEVELS)
    g = ctx.solve(inst, R, 0.0, tmax, fixed_sweeps=1, m0=m0, t0=t0,
                  outputs=("m_final", "sweeps", "levels"))
    o = O.mars_solve(O.Instance.dense(J), m0, t0, fixed_sweeps=1)
    check_trajectory(g.m_final, o["m"], "strict")
    assert np.array_equal(g.replica_sweeps, o["sweeps"])
    assert np.array_equal(g.replica_levels, o["levels"])
    ctx.free(inst)


@pytest.mark.parametrize("n", [8000, 9000, 12000, 14402])
def test_large_n_kernel_choice(ctx, n):
    J = I.sk_gauss(n, 11)
    inst = ctx.add_dense(J)
    R, tmax, c = 5, 2.0, 0.25
    m0, t0 = I.replica_inputs(R, n, 0.0, tmax, 31)
    t0 = floored_t0(t0, c, max_levels=STRICT_LEVELS)
    g = ctx.solve(inst, R, 0.0, tmax, c_step=c, fixed_sweeps=1, m0=m0, t0=t0,
                  outputs=("m_final", "sweeps", "energies", "spins"))
    oi = O.Instance.dense(J)
    o = O.mars_solve(oi, m0, t0, c_step=c, fixed_sweeps=1)
    check_trajectory(g.m_final, o["m"], "strict")
    assert np.array_equal(g.replica_sweeps, o["sweeps"])
    assert np.array_equal(g.energies, O.energies(oi, g.spins))
    ctx.free(inst)
