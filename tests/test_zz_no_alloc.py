"""mars_solve_noalloc against mars_solve, through the C ABI, on the GPU.

mars_solve_noalloc exists for callers that cannot allocate device memory
while they run: a host program whose device memory is fully reserved up front
by another framework's allocator, or a latency-bound loop that must not call
an allocator (or risk its failure) once it has started. It keeps every
per-solve buffer in one static device array, so this test checks that its
results equal those of the allocating entry point on the same inputs, on two
calls in a row (the second call reuses the array the first one left behind),
and that a warm call takes no device memory: neither from the device's
stream-ordered pool (which the allocating entry point draws on) nor through
cudaMalloc, as the CUDA driver reports them.
"""
import ctypes

import numpy as np
import pytest

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


def _noalloc(ctx, inst, n, R, seed, t_max):
    import torch
    from paper_1907_05124_gb300 import mars
    p = mars.Params()
    ctx._lib.mars_params_default(ctypes.byref(p))
    p.replicas, p.t_min, p.t_max, p.seed = R, 0.0, t_max, seed
    best = torch.zeros(n, dtype=torch.int8, device="cuda")
    energies = torch.zeros(R, dtype=torch.float64, device="cuda")
    res = mars.Result()
    torch.cuda.synchronize()
    rc = ctx._lib.mars_solve_noalloc(ctx._ctx, inst, ctypes.byref(p), best.data_ptr(),
                                     energies.data_ptr(), ctypes.byref(res))
    return rc, best.cpu().numpy(), energies.cpu().numpy(), res


@pytest.mark.parametrize("kind", ["lattice", "dense"])
def test_noalloc_matches_solve_on_two_calls(ctx, kind):
    if kind == "lattice":
        csr = I.ea_lattice(24, 2, 3)
        inst, n, t_max = ctx.add_csr(*csr), csr.n, 4.0
    else:
        J = I.sk_pm1(48, 1)
        inst, n, t_max = ctx.add_dense(J), 48, 12.0
    R = 96
    for seed in (11, 12):  # two calls in a row share the static array
        ref = ctx.solve(inst, R, 0.0, t_max, seed=seed, outputs=("energies",))
        rc, best, energies, res = _noalloc(ctx, inst, n, R, seed, t_max)
        assert rc == 0, ctx._lib.mars_last_error(ctx._ctx).decode()
        # integer couplings: energies are exact, so the tolerance is zero
        assert np.array_equal(energies, ref.energies)
        assert res.best_energy == ref.best_energy
        assert res.best_replica == ref.best_replica and res.hits == ref.hits
        assert res.sweeps == ref.sweeps
        assert np.array_equal(best, ref.best_spins)
    ctx.free(inst)


def test_noalloc_rejects_work_beyond_the_static_limit(ctx):
    from paper_1907_05124_gb300 import mars
    csr = I.ea_lattice(100, 2, 0)
    inst = ctx.add_csr(*csr)
    R = (mars.NOALLOC_SCRATCH_BYTES // csr.n) + 1  # R*n spins alone exceed the array
    rc, _, _, _ = _noalloc(ctx, inst, csr.n, R, 0, 4.0)
    assert rc == mars.MARS_EINVAL
    assert b"static limit" in ctx._lib.mars_last_error(ctx._ctx)
    ctx.free(inst)


class _DeviceMemory:
    """What the CUDA driver reports about device memory: the default
    stream-ordered pool's bytes in use (and their high-water mark since the
    last reset), and the device's free bytes."""

    _USED_CURRENT, _USED_HIGH = 7, 8  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT / _HIGH

    def __init__(self, ordinal):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), ordinal) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _attr(self, a):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, a, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self._USED_HIGH, ctypes.byref(zero)) == 0

    def snapshot(self):
        free, total = ctypes.c_size_t(), ctypes.c_size_t()
        assert self.cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
        return self._attr(self._USED_CURRENT), self._attr(self._USED_HIGH), free.value


def test_noalloc_takes_no_device_memory(ctx):
    """A warm call allocates nothing: the pool's high-water mark stays at what
    was in use before the calls and the device's free memory is unchanged,
    while the allocating entry point, measured the same way, does move the
    pool's high-water mark (so the measurement can see an allocation)."""
    import torch
    from paper_1907_05124_gb300 import mars
    csr = I.ea_lattice(24, 2, 5)
    inst, n, R = ctx.add_csr(*csr), csr.n, 64
    p = mars.Params()
    ctx._lib.mars_params_default(ctypes.byref(p))
    p.replicas, p.t_min, p.t_max, p.seed = R, 0.0, 4.0, 3
    best = torch.zeros(n, dtype=torch.int8, device="cuda")
    energies = torch.zeros(R, dtype=torch.float64, device="cuda")
    res = mars.Result()

    def call():
        rc = ctx._lib.mars_solve_noalloc(ctx._ctx, inst, ctypes.byref(p), best.data_ptr(),
                                         energies.data_ptr(), ctypes.byref(res))
        assert rc == 0, ctx._lib.mars_last_error(ctx._ctx).decode()

    call()  # warm: the first call looks up the static array's address
    torch.cuda.synchronize()
    mem = _DeviceMemory(torch.cuda.current_device())
    used0, _, free0 = mem.snapshot()
    mem.reset_high()
    call()
    call()
    torch.cuda.synchronize()
    used1, high1, free1 = mem.snapshot()
    assert high1 <= used0 and used1 == used0, (used0, high1, used1)
    assert free1 == free0, (free0, free1)
    # the probe sees the allocating entry point's buffers
    mem.reset_high()
    ctx.solve(inst, R, 0.0, 4.0, seed=3)
    torch.cuda.synchronize()
    _, high2, _ = mem.snapshot()
    assert high2 > used0
    ctx.free(inst)
