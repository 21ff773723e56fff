"""Failure detection, with every failure made on the host (no GPU fault).

* A device-side wait with a budget: mars_device_check's kernel polls a flag
  in host-mapped memory; with MARS_FAULT=flag the host never raises it, the
  wait runs out, MARS_ETIMEOUT reaches the caller and the context keeps
  working.
* An injected allocation failure (MARS_FAULT=alloc:K) surfaces as
  MARS_ENOMEM from the call that made the K-th allocation, leaves nothing
  half-registered, and later calls succeed with the same results.
* A cancelled request: dropped while queued, or its results discarded after
  it ran; mars_poll reports MARS_ECANCELED and the other requests are
  unaffected.
"""
import time

import numpy as np
import pytest

from paper_1907_05124_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mars():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05124_gb300 import build, mars as m
    build.build()
    return m


def _same(a, b):
    assert a.best_energy == b.best_energy and a.best_replica == b.best_replica
    assert a.sweeps == b.sweeps and np.array_equal(a.best_spins, b.best_spins)


def test_device_check_sees_the_flag(mars):
    with mars.Context(0) as c:
        for _ in range(3):
            c.device_check(1_000_000)


def test_device_wait_runs_out_and_context_stays_usable(mars, monkeypatch):
    csr = I.ea_lattice(12, 2, 1)
    with mars.Context(0) as ref:
        want = ref.solve(ref.add_csr(*csr), 32, 0.0, 4.0, seed=3)
    monkeypatch.setenv("MARS_FAULT", "flag")
    with mars.Context(0) as c:
        monkeypatch.delenv("MARS_FAULT")
        t = time.time()
        with pytest.raises(mars.MarsError) as e:
            c.device_check(2000)  # 2 ms
        assert e.value.code == mars.MARS_ETIMEOUT
        assert time.time() - t < 5.0
        # the context keeps working after the device gave up
        _same(c.solve(c.add_csr(*csr), 32, 0.0, 4.0, seed=3), want)
        with pytest.raises(mars.MarsError):
            c.device_check(0)  # budget out of range


def test_injected_allocation_failure(mars, monkeypatch):
    csr = I.ea_lattice(12, 2, 2)
    with mars.Context(0) as ref:
        want = ref.solve(ref.add_csr(*csr), 24, 0.0, 4.0, seed=5)
    # the smallest K whose failure lets registration through: K - 1 allocations register
    k = 1
    while True:
        monkeypatch.setenv("MARS_FAULT", f"alloc:{k}")
        with mars.Context(0) as c:
            try:
                c.add_csr(*csr)
                break
            except mars.MarsError as e:
                assert e.code == mars.MARS_ENOMEM
        k += 1
        assert k < 64
    monkeypatch.setenv("MARS_FAULT", f"alloc:{k}")
    with mars.Context(0) as c:
        monkeypatch.delenv("MARS_FAULT")
        inst = c.add_csr(*csr)  # K - 1 allocations: fine
        with pytest.raises(mars.MarsError) as e:
            c.solve(inst, 24, 0.0, 4.0, seed=5)  # its first allocation is the K-th
        assert e.value.code == mars.MARS_ENOMEM and b"MARS_FAULT" in c._lib.mars_last_error(c._ctx)
        _same(c.solve(inst, 24, 0.0, 4.0, seed=5), want)
    # registration that fails leaves no instance behind
    monkeypatch.setenv("MARS_FAULT", "alloc:1")
    with mars.Context(0) as c:
        monkeypatch.delenv("MARS_FAULT")
        with pytest.raises(mars.MarsError):
            c.add_csr(*csr)
        inst = c.add_csr(*csr)
        _same(c.solve(inst, 24, 0.0, 4.0, seed=5), want)


def _poll(c, r, timeout=120.0):
    t = time.time()
    while True:
        res = c.poll(r)
        if res is not None:
            return res
        assert time.time() - t < timeout
        time.sleep(0.001)


def test_cancel_queued_and_running_requests(mars):
    with mars.Context(0) as c:
        big = c.add_csr(*I.ea_lattice(80, 2, 3))
        small = c.add_csr(*I.er_graph(600, 8, 4, "pm1"))
        dense = c.add_dense(I.sk_gauss(512, 5))
        c.serve_limits(1)  # one at a time: the later ones queue
        running = c.submit(big, 2048, 0.0, 4.0, seed=1)
        queued = c.submit(small, 64, 0.0, 6.0, seed=2)
        kept = c.submit(small, 64, 0.0, 6.0, seed=3)
        c.cancel(queued)
        c.cancel(running)
        for r in (queued, running):
            with pytest.raises(mars.MarsError) as e:
                _poll(c, r)
            assert e.value.code == mars.MARS_ECANCELED
        _same(_poll(c, kept), c.solve(small, 64, 0.0, 6.0, seed=3))
        # a tensor-core request stops after its current batch of sweeps
        tc = c.submit(dense, 256, 0.0, 2.0, c_step=1 / 512 ** 0.5, precision="bf16", seed=4)
        time.sleep(0.05)
        c.cancel(tc)
        with pytest.raises(mars.MarsError) as e:
            _poll(c, tc)
        assert e.value.code == mars.MARS_ECANCELED
        assert c.serve_status() == (0, 0)
        with pytest.raises(mars.MarsError):
            c.cancel(12345)  # unknown id
