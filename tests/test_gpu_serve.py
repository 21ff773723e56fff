"""Serving: requests submitted while others run give the results they give alone.

Every replica of a served request computes exactly what it computes in a
blocking mars_solve with the same parameters (the replica order differs, the
arithmetic does not), so each served request's best energy, best replica,
hits and sweep counts must equal the blocking solve's, whatever else was in
flight on the GPU at the time.
"""
import time

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


def _wait(ctx, reqs, timeout=300.0):
    out, t0 = {}, time.time()
    while len(out) < len(reqs):
        for r in reqs:
            if r not in out:
                res = ctx.poll(r)
                if res is not None:
                    out[r] = res
        assert time.time() - t0 < timeout, "served requests did not finish"
        time.sleep(0.001)
    return out


def _same(a, b):
    assert a.best_energy == b.best_energy
    assert a.best_replica == b.best_replica
    assert a.hits == b.hits
    assert a.sweeps == b.sweeps and a.levels == b.levels and a.capped_levels == b.capped_levels
    assert np.array_equal(a.best_spins, b.best_spins)


def test_mixed_requests_match_blocking_solves(ctx):
    graphs = {"lat": I.ea_lattice(40, 2, 1), "er": I.er_graph(2000, 8, 2, "pm1"),
              "er_one": I.er_graph(800, 20, 3, "one"), "lat3": I.ea_lattice(10, 3, 4)}
    insts = {k: ctx.add_csr(*g) for k, g in graphs.items()}
    sk = I.sk_pm1(96, 5)
    insts["sk"] = ctx.add_dense(sk)
    gauss = I.sk_gauss(256, 6)
    insts["sk_bf16"] = ctx.add_dense(gauss)
    big = I.sk_gauss(4096, 7)  # a tensor-core request at N = 4096 in the mix
    insts["sk4096_bf16"] = ctx.add_dense(big)
    plan = [("lat", 200, 4.0, {}), ("er", 64, 6.0, {}), ("sk", 128, 20.0, {}),
            ("er_one", 96, 10.0, {}), ("lat3", 50, 5.0, {}), ("lat", 33, 4.0, {}),
            ("sk_bf16", 64, 2.0, {"precision": "bf16", "c_step": 1 / 16.0}), ("er", 7, 6.0, {}),
            ("sk4096_bf16", 96, 0.4, {"precision": "bf16", "c_step": 1 / 64.0})]
    ctx.serve_limits(4)  # fewer slots than requests: some wait for a slot
    reqs = []
    for j, (k, R, tmax, kw) in enumerate(plan):
        reqs.append(ctx.submit(insts[k], R, 0.0, tmax, seed=100 + j, **kw))
    served = _wait(ctx, reqs)
    for j, (k, R, tmax, kw) in enumerate(plan):
        ref = ctx.solve(insts[k], R, 0.0, tmax, seed=100 + j, **kw)
        _same(served[reqs[j]], ref)
    # exact energies of the returned spins
    r0 = served[reqs[0]]
    assert r0.best_energy == O.energy(O.Instance.csr(graphs["lat"]), r0.best_spins)
    r6 = served[reqs[6]]
    assert r6.best_energy == O.energy(O.Instance.dense(gauss), r6.best_spins)
    r8 = served[reqs[8]]
    assert r8.best_energy == O.energy(O.Instance.dense(big), r8.best_spins)
    assert ctx.serve_status() == (0, 0)
    for i in insts.values():
        ctx.free(i)


def test_budget_admission_and_oversized_request():
    torch = pytest.importorskip("torch")
    from paper_1907_05124_gb300 import mars
    from paper_1907_05124_gb300.mars import MarsError, MARS_ENOMEM
    c = mars.Context(0, hbm_budget_bytes=24 << 20)
    g = I.ea_lattice(30, 2, 0)
    inst = c.add_csr(*g)
    small = [c.submit(inst, 256, 0.0, 4.0, seed=s) for s in range(6)]
    big = c.submit(inst, 40000, 0.0, 4.0, seed=9)  # ~36 MB of spins: can never fit
    done = _wait(c, small)
    assert len(done) == 6
    with pytest.raises(MarsError) as e:
        while c.poll(big) is None:
            time.sleep(0.001)
    assert e.value.code == MARS_ENOMEM
    c.close()


def _serve_once(budget, g, R, kw):
    """Serve one request in a fresh context with the given HBM budget:
    True when it ran, False when it was refused for memory."""
    from paper_1907_05124_gb300 import mars
    from paper_1907_05124_gb300.mars import MarsError, MARS_ENOMEM
    c = mars.Context(0, hbm_budget_bytes=budget)
    try:
        try:
            inst = c.add_csr(*g)
            r = c.submit(inst, R, 0.0, 6.0, seed=3, **kw)
            while c.poll(r) is None:
                time.sleep(0.001)
            return True
        except MarsError as e:
            if e.code == MARS_ENOMEM:
                return False
            raise
    finally:
        c.close()


def test_tight_budget_request_waits_instead_of_failing(ctx):
    """Admission counts everything a request will allocate. Under a budget
    that holds exactly one synchronous (Jacobi) request, whose second buffer
    of magnetisations is plan-dependent scratch, a second such request waits
    for the first to finish instead of failing half-way through its set-up."""
    from paper_1907_05124_gb300 import mars
    g = I.er_graph(3000, 10, 41, "pm1")
    R, kw = 96, {"update": "jacobi", "k_max": 400}  # synchronous sweeps cycle: every level capped
    lo, hi = 1 << 20, 1 << 30
    assert _serve_once(hi, g, R, kw)
    while hi - lo > (64 << 10):  # the smallest budget one request runs under
        mid = (lo + hi) // 2
        if _serve_once(mid, g, R, kw):
            hi = mid
        else:
            lo = mid
    c = mars.Context(0, hbm_budget_bytes=hi)
    try:
        inst = c.add_csr(*g)
        reqs = [c.submit(inst, R, 0.0, 6.0, seed=3 + k, **kw) for k in range(3)]
        queued, running = c.serve_status()
        assert running <= 1 and queued >= 1  # the budget holds one at a time
        out = _wait(c, reqs)  # raises if any of them failed
    finally:
        c.close()
    ref_inst = ctx.add_csr(*g)
    for k, r in enumerate(reqs):
        _same(out[r], ctx.solve(ref_inst, R, 0.0, 6.0, seed=3 + k, **kw))
    ctx.free(ref_inst)


def test_poll_unknown_request(ctx):
    from paper_1907_05124_gb300.mars import MarsError
    ctx._req_n = getattr(ctx, "_req_n", {})
    ctx._req_n[123456] = 4
    with pytest.raises(MarsError):
        ctx.poll(123456)


def test_ring_joins_running_launch_and_matches_blocking(ctx):
    """Continuous batching into the persistent kernel: sparse integer requests
    are published into the serving ring; requests submitted while a long one
    runs join the same launch. Every result equals the blocking solve's."""
    big = ctx.add_csr(*I.ea_lattice(60, 2, 11))
    smalls = [ctx.add_csr(*g) for g in (I.er_graph(700, 6, 12, "pm1"), I.ea_lattice(20, 2, 13),
                                          I.er_graph(1500, 10, 14, "one"), I.ea_lattice(8, 3, 15))]
    ring0, _ = ctx.serve_counters()
    reqs = {ctx.submit(big, 2048, 0.0, 4.0, seed=21): (big, 2048, 4.0, 21)}
    time.sleep(0.002)  # the big job is on the GPU when the next ones arrive
    for j, inst in enumerate(smalls):
        for rep in range(3):
            sd = 100 + 10 * j + rep
            reqs[ctx.submit(inst, 96 + 32 * rep, 0.0, 5.0, seed=sd)] = (inst, 96 + 32 * rep, 5.0, sd)
    out = _wait(ctx, list(reqs))
    ring1, _ = ctx.serve_counters()
    assert ring1 - ring0 == len(reqs)  # every one of these went through the ring
    for r, (inst, R, tmax, sd) in reqs.items():
        _same(out[r], ctx.solve(inst, R, 0.0, tmax, seed=sd))
    for inst in [big] + smalls:
        ctx.free(inst)


def test_ring_kernel_relaunches_after_idle_exit(ctx):
    """The serving kernel exits after about 100 us without work; a request
    submitted later starts it again, and the ring resets once it is idle."""
    inst = ctx.add_csr(*I.ea_lattice(16, 2, 17))
    for wave in range(3):
        reqs = [ctx.submit(inst, 64, 0.0, 4.0, seed=wave * 10 + k) for k in range(4)]
        out = _wait(ctx, reqs)
        for k, r in enumerate(reqs):
            _same(out[r], ctx.solve(inst, 64, 0.0, 4.0, seed=wave * 10 + k))
        time.sleep(0.05)
    ctx.free(inst)


def test_ring_takes_large_instances_with_one_slot(ctx):
    """An instance whose two replicas' magnetisations do not fit on chip runs
    in the serving ring with one slot per CTA, beside two-slot jobs."""
    big = ctx.add_csr(*I.ea_lattice(32, 3, 25))
    small = ctx.add_csr(*I.ea_lattice(20, 2, 26))
    ring0, _ = ctx.serve_counters()
    reqs = {ctx.submit(big, 40, 0.0, 6.0, seed=1): (big, 40, 6.0, 1),
            ctx.submit(small, 100, 0.0, 4.0, seed=2): (small, 100, 4.0, 2)}
    out = _wait(ctx, list(reqs))
    assert ctx.serve_counters()[0] - ring0 == 2
    for r, (inst, R, tmax, sd) in reqs.items():
        _same(out[r], ctx.solve(inst, R, 0.0, tmax, seed=sd))
    ctx.free(big)
    ctx.free(small)


def test_served_quench_matches_blocking(ctx):
    inst = ctx.add_csr(*I.er_graph(800, 8, 29, "pm1"))
    r = ctx.submit(inst, 64, 0.0, 5.0, seed=9, quench=True, geometric=0.75, t_floor=0.5)
    out = _wait(ctx, [r])
    _same(out[r], ctx.solve(inst, 64, 0.0, 5.0, seed=9, quench=True, geometric=0.75, t_floor=0.5))
    ctx.free(inst)


def test_ring_jobs_pass_queued_dense_requests():
    """Admission by class: with one in-flight slot for the other requests, a
    dense tensor-core request runs and a second one waits for the slot; a
    small sparse request submitted after both runs at once as a job of the
    persistent serving kernel and finishes first. Every result equals its
    blocking solve."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05124_gb300 import build, mars
    build.build()
    c = mars.Context(0)
    try:
        dense = c.add_dense(I.sk_gauss(2048, 21))
        lat = c.add_csr(*I.ea_lattice(32, 2, 22))
        c.serve_limits(1)
        kw = {"precision": "bf16", "c_step": 1 / 32.0}
        d1 = c.submit(dense, 256, 0.0, 2.0, seed=1, **kw)
        d2 = c.submit(dense, 256, 0.0, 2.0, seed=2, **kw)
        small = c.submit(lat, 64, 0.0, 4.0, seed=3)
        done, order, t0 = {}, [], time.time()
        while len(done) < 3:
            for r in (d1, d2, small):
                if r not in done:
                    res = c.poll(r)
                    if res is not None:
                        done[r] = res
                        order.append(r)
            assert time.time() - t0 < 300.0, "served requests did not finish"
            time.sleep(0.0005)
        assert order[0] == small and order.index(d1) < order.index(d2)
        _same(done[d1], c.solve(dense, 256, 0.0, 2.0, seed=1, **kw))
        _same(done[d2], c.solve(dense, 256, 0.0, 2.0, seed=2, **kw))
        _same(done[small], c.solve(lat, 64, 0.0, 4.0, seed=3))
        assert c.serve_status() == (0, 0)
    finally:
        c.close()
