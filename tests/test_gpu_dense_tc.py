"""Dense tensor-core path (precision BF16) against the FP64 oracle.

The BF16 path computes each 128-spin panel's fields with a tcgen05 GEMM over
BF16 copies of J and of the magnetisations, then updates the panel's spins in
sequence in FP32. Two kinds of checks:

* exact structure: with J block-diagonal in 128-spin blocks (+-1 inside) and
  start states exactly representable in BF16, every panel's GEMM sees only
  BF16-exact inputs, so one sweep must equal the sequential FP64 sweep to FP32
  rounding (max-abs 1e-5). A wrong TMA coordinate, descriptor, swizzle or
  split-K reduction breaks this.
* full instances: BF16 rounding of updated spins moves trajectories, so the
  bar is the method's outcome: every returned energy is the exact energy of
  the returned spins, and the energy distribution matches the oracle's.
"""
import numpy as np
import pytest

import oracle as O
from paper_1907_05124_gb300 import instances as I
from test_gpu_parity import SENS_FACTOR, record_long_tier

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


def block_diagonal_pm1(n, seed, block=128):
    rng = np.random.default_rng(seed)
    J = np.zeros((n, n))
    for b0 in range(0, n, block):
        b1 = min(n, b0 + block)
        k = b1 - b0
        u = np.triu(rng.choice(np.array([-1.0, 1.0]), size=(k, k)), 1)
        J[b0:b1, b0:b1] = u + u.T
    return J


def bf16_exact_m0(R, n, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(-128, 129, size=(R, n)) / 128.0).astype(np.float32)


def _sensitivity(inst, m0, t0, **kw):
    rng = np.random.default_rng(99)
    bumped = np.nextafter(m0, np.where(rng.random(m0.shape) < 0.5, -2.0, 2.0).astype(np.float32))
    a = O.mars_solve(inst, m0, t0, **kw)["m"]
    b = O.mars_solve(inst, bumped, t0, **kw)["m"]
    return float(np.abs(a - b).max())


@pytest.mark.parametrize("regime", ["contracting", "saturated"])
@pytest.mark.parametrize("n,R,with_h", [(512, 200, False), (320, 130, True), (128, 64, False),
                                         (1024, 300, False)])
def test_block_diagonal_sweep(ctx, n, R, with_h, regime):
    """One sweep over block-diagonal +-1 J with BF16-exact start states.

    contracting: one level at T in [24, 28), above the blocks' spectral edge
    (about 2 sqrt(128) = 22.6), where the sequential map contracts and an ideal
    FP32 sweep stays within 1e-7 of FP64: the bar is the strict 1e-5.
    saturated: T in [0.5, 1), where rounding is amplified along the 128-spin
    chain (an ideal FP32 sweep already differs by ~5e-5); the bar is 1e-5 plus
    50 times the oracle's own change under a one-ulp perturbation of m0.
    """
    J = block_diagonal_pm1(n, n)
    h = np.random.default_rng(1).integers(-2, 3, size=n).astype(np.float64) if with_h else None
    inst = ctx.add_dense(J, h=h)
    m0 = bf16_exact_m0(R, n, 3)
    rng = np.random.default_rng(4)
    if regime == "contracting":
        c, t0 = 30.0, rng.uniform(54.0, 58.0, size=R).astype(np.float32)
    else:
        c, t0 = 1.0, rng.uniform(1.5, 2.0, size=R).astype(np.float32)
    g = ctx.solve(inst, R, float(t0.min()), float(t0.max()), c_step=c, fixed_sweeps=1, m0=m0,
                  t0=t0, precision="bf16", outputs=("m_final", "energies", "spins", "sweeps"))
    oi = O.Instance.dense(J, h)
    o = O.mars_solve(oi, m0, t0, c_step=c, fixed_sweeps=1)
    err = np.abs(g.m_final - o["m"]).max()
    if regime == "contracting":
        assert err <= 1e-5, err
    else:
        delta = _sensitivity(oi, m0, t0, c_step=c, fixed_sweeps=1)
        record_long_tier(float(err), delta)
        assert err <= 1e-5 + SENS_FACTOR * delta, (err, delta)
    assert np.array_equal(g.replica_sweeps, o["sweeps"])
    assert np.array_equal(g.energies, O.energies(oi, g.spins))
    ctx.free(inst)


def test_sk_pm1_energies_exact_and_distribution(ctx):
    from scipy import stats
    n, R = 256, 384
    J = I.sk_pm1(n, 7)
    inst = ctx.add_dense(J)
    m0, t0 = I.replica_inputs(R, n, 0.0, 32.0, 8)
    g = ctx.solve(inst, R, 0.0, 32.0, m0=m0, t0=t0, precision="bf16",
                  outputs=("energies", "spins", "sweeps"))
    oi = O.Instance.dense(J)
    assert np.array_equal(g.energies, O.energies(oi, g.spins))
    assert g.best_energy == O.energy(oi, g.best_spins)
    o = O.mars_solve(oi, m0, t0, nthreads=8, want_m=False)
    assert stats.ks_2samp(g.energies, o["energy"]).pvalue > 0.01
    # same quality: best energies within 1 % of each other
    assert abs(g.best_energy - o["energy"].min()) <= 0.01 * abs(o["energy"].min())
    ctx.free(inst)


def test_sk_gaussian_energies(ctx):
    n, R = 384, 96
    J = I.sk_gauss(n, 5)
    inst = ctx.add_dense(J)
    c = float(1.0 / np.sqrt(n))
    m0, t0 = I.replica_inputs(R, n, 0.0, 2.0, 6)
    g = ctx.solve(inst, R, 0.0, 2.0, c_step=c, fixed_sweeps=2, m0=m0, t0=t0, precision="bf16",
                  outputs=("energies", "spins", "levels"))
    oi = O.Instance.dense(J)
    assert np.array_equal(g.energies, O.energies(oi, g.spins))  # FP64 bit-exact
    o = O.mars_solve(oi, m0, t0, c_step=c, fixed_sweeps=2, nthreads=8, want_m=False)
    assert np.array_equal(g.replica_levels, o["levels"])
    assert abs(g.best_energy - o["energy"].min()) <= 0.02 * abs(o["energy"].min())
    ctx.free(inst)


def test_bf16_rejected_where_not_available(ctx):
    from paper_1907_05124_gb300.mars import MarsError
    inst = ctx.add_csr(*I.ea_lattice(8, 2, 0))
    with pytest.raises(MarsError):
        ctx.solve(inst, 4, 0.0, 4.0, precision="bf16")
    ctx.free(inst)
    dinst = ctx.add_dense(I.sk_pm1(64, 0))
    with pytest.raises(MarsError):
        ctx.solve(dinst, 4, 0.0, 4.0, precision="bf16", update="jacobi")
    ctx.free(dinst)


def test_fp32_polish_leaves_fixed_points(ctx):
    """After a BF16 descent with the FP32 polish, every replica that converged
    its last level sits at a fixed point of the update at that temperature:
    ||m + tanh((J m + h)/T)||_inf <= d_min ||J||_inf / T (the bound the oracle
    pins), up to FP32 rounding of m."""
    n, R, c = 256, 32, 1.0 / 16.0
    J = I.sk_gauss(n, 11)
    inst = ctx.add_dense(J)
    g = ctx.solve(inst, R, 0.0, 2.0, c_step=c, precision="bf16", polish=True,
                  outputs=("m_final", "t0", "levels", "energies", "spins", "capped"))
    jinf = np.abs(J).sum(axis=1).max()
    checked = 0
    for r in range(R):
        if g.replica_levels[r] == 0 or g.replica_capped[r] > 0:
            continue
        T = float(g.t0[r])
        for _ in range(int(g.replica_levels[r])):
            T = T - c
        m = g.m_final[r].astype(np.float64)
        resid = np.abs(m + np.tanh(J @ m / T)).max()
        assert resid <= 1e-4 * jinf / T + 1e-5, (r, resid)
        checked += 1
    assert checked >= R // 2
    assert np.array_equal(g.energies, O.energies(O.Instance.dense(J), g.spins))
    ctx.free(inst)


def block_tridiagonal_pm1(n, seed, block=128):
    rng = np.random.default_rng(seed)
    u = np.triu(rng.choice(np.array([-1.0, 1.0]), size=(n, n)), 1)
    b = np.arange(n) // block
    u *= np.abs(b[:, None] - b[None, :]) <= 1
    return u + u.T


@pytest.mark.parametrize("n,R", [(640, 256), (600, 72)])
def test_overlapped_panels_block_tridiagonal(ctx, monkeypatch, n, R):
    """Panel p+1's GEMM leaves panel p out and runs beside panel p's chain,
    which adds panel p's new spins to panel p+1's fields in FP32.

    With J block-tridiagonal in 128-spin blocks (+-1 inside) and BF16-exact
    start states, every field of the first sweep is then assembled from exact
    BF16 products (old spins) and FP32 products (the previous panel's new
    spins), so in the contracting regime (one level, T in [50, 54), above the
    spectral edge 2 sqrt(3 * 128) = 39) one sweep equals the FP64 sweep to
    1e-5. The plain sweep, which passes the previous panel's new spins through
    the BF16 GEMM, misses that bar (an FP64 emulation of it errs by 2e-4), so
    the test also shows that the overlapped path ran. The chain must give
    bit-identical results for 1, 2 and 4 replicas per warp.
    """
    J = block_tridiagonal_pm1(n, 3)
    inst = ctx.add_dense(J)
    m0 = bf16_exact_m0(R, n, 5)
    t0 = np.random.default_rng(6).uniform(110.0, 114.0, size=R).astype(np.float32)
    oi = O.Instance.dense(J)
    o = O.mars_solve(oi, m0, t0, c_step=60.0, fixed_sweeps=1)
    assert np.all(o["levels"] == 1)
    kw = dict(c_step=60.0, fixed_sweeps=1, m0=m0, t0=t0, precision="bf16",
              outputs=("m_final", "energies", "spins"))
    monkeypatch.setenv("MARS_TC_OVERLAP", "0")
    plain = ctx.solve(inst, R, float(t0.min()), float(t0.max()), **kw)
    assert np.abs(plain.m_final - o["m"]).max() > 1e-5
    monkeypatch.setenv("MARS_TC_OVERLAP", "1")
    runs = {}
    for rpw in (1, 2, 4):
        monkeypatch.setenv("MARS_TC_RPW", str(rpw))
        runs[rpw] = ctx.solve(inst, R, float(t0.min()), float(t0.max()), **kw)
    err = np.abs(runs[1].m_final - o["m"]).max()
    assert err <= 1e-5, err
    for rpw in (2, 4):
        assert np.array_equal(runs[rpw].m_final, runs[1].m_final), rpw
        assert np.array_equal(runs[rpw].energies, runs[1].energies)
    assert np.array_equal(runs[1].energies, O.energies(oi, runs[1].spins))
    ctx.free(inst)


def test_overlap_and_plain_sweeps_reach_the_same_quality(ctx, monkeypatch):
    """The overlapped sweep (previous panel in FP32) and the plain one (all of
    J through the BF16 GEMM) are two roundings of the same method: on an SK
    instance both return exact energies and best energies within 1 % of the
    oracle's."""
    n, R = 512, 256
    J = I.sk_pm1(n, 12)
    inst = ctx.add_dense(J)
    m0, t0 = I.replica_inputs(R, n, 0.0, 48.0, 13)
    oi = O.Instance.dense(J)
    o = O.mars_solve(oi, m0, t0, nthreads=8, want_m=False)
    for ov in ("0", "1"):
        monkeypatch.setenv("MARS_TC_OVERLAP", ov)
        g = ctx.solve(inst, R, 0.0, 48.0, m0=m0, t0=t0, precision="bf16", outputs=("energies", "spins"))
        assert np.array_equal(g.energies, O.energies(oi, g.spins))
        assert abs(g.best_energy - o["energy"].min()) <= 0.01 * abs(o["energy"].min()), ov
    ctx.free(inst)


def fp8_exact_m0(R, n, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(-8, 9, size=(R, n)) / 8.0).astype(np.float32)


@pytest.mark.parametrize("n,R", [(512, 200), (320, 130), (1024, 300)])
def test_fp8_block_diagonal_sweep(ctx, n, R):
    """E4M3 operands (tcgen05 kind::f8f6f4). With block-diagonal +-1 J and
    start states k/8 (exact in E4M3) every panel GEMM sees exact inputs, so in
    the contracting regime (one level, T in [24, 28)) one sweep equals the
    sequential FP64 sweep to 1e-5. A wrong instruction descriptor, K step or
    tensor map breaks this."""
    J = block_diagonal_pm1(n, n)
    inst = ctx.add_dense(J)
    m0 = fp8_exact_m0(R, n, 3)
    t0 = np.random.default_rng(4).uniform(54.0, 58.0, size=R).astype(np.float32)
    g = ctx.solve(inst, R, float(t0.min()), float(t0.max()), c_step=30.0, fixed_sweeps=1, m0=m0, t0=t0,
                  precision="fp8", outputs=("m_final", "energies", "spins", "sweeps"))
    oi = O.Instance.dense(J)
    o = O.mars_solve(oi, m0, t0, c_step=30.0, fixed_sweeps=1)
    err = np.abs(g.m_final - o["m"]).max()
    assert err <= 1e-5, err
    assert np.array_equal(g.replica_sweeps, o["sweeps"])
    assert np.array_equal(g.energies, O.energies(oi, g.spins))
    ctx.free(inst)


def test_fp8_overlapped_panels_block_tridiagonal(ctx, monkeypatch):
    """The overlapped sweep with E4M3 operands: the GEMM leaves one 128-wide
    K block (one panel) out, and the previous panel's part of the fields is
    FP32, so one contracting sweep equals the FP64 sweep to 1e-5, for every
    replicas-per-warp choice alike."""
    n, R = 640, 200
    J = block_tridiagonal_pm1(n, 5)
    inst = ctx.add_dense(J)
    m0 = fp8_exact_m0(R, n, 6)
    t0 = np.random.default_rng(7).uniform(110.0, 114.0, size=R).astype(np.float32)
    oi = O.Instance.dense(J)
    o = O.mars_solve(oi, m0, t0, c_step=60.0, fixed_sweeps=1)
    kw = dict(c_step=60.0, fixed_sweeps=1, m0=m0, t0=t0, precision="fp8", outputs=("m_final",))
    monkeypatch.setenv("MARS_TC_OVERLAP", "1")
    runs = []
    for rpw in (1, 2, 4):
        monkeypatch.setenv("MARS_TC_RPW", str(rpw))
        runs.append(ctx.solve(inst, R, float(t0.min()), float(t0.max()), **kw))
    assert np.abs(runs[0].m_final - o["m"]).max() <= 1e-5
    for r in runs[1:]:
        assert np.array_equal(r.m_final, runs[0].m_final)
    ctx.free(inst)


def test_fp8_rejected_where_not_exact(ctx):
    from paper_1907_05124_gb300.mars import MarsError
    g = ctx.add_dense(I.sk_gauss(64, 1))
    with pytest.raises(MarsError):
        ctx.solve(g, 4, 0.0, 1.0, precision="fp8")
    ctx.free(g)
    J = I.sk_pm1(64, 2) * 17.0  # 17 needs four mantissa bits
    d = ctx.add_dense(J)
    with pytest.raises(MarsError):
        ctx.solve(d, 4, 0.0, 1.0, precision="fp8")
    ctx.free(d)
    s = ctx.add_csr(*I.ea_lattice(6, 2, 0))
    with pytest.raises(MarsError):
        ctx.solve(s, 4, 0.0, 4.0, precision="fp8")
    ctx.free(s)


def test_fp8_sk_pm1_quality(ctx):
    """E4M3 magnetisation copies keep three mantissa bits, so trajectories move
    further than with BF16; the bar is the method's outcome: exact energies of
    the returned spins and a best energy within 1 % of the oracle's (a GB300
    run of this instance found -8650 against the oracle's -8648)."""
    n, R = 512, 256
    J = I.sk_pm1(n, 7)
    inst = ctx.add_dense(J)
    m0, t0 = I.replica_inputs(R, n, 0.0, 48.0, 8)
    oi = O.Instance.dense(J)
    o = O.mars_solve(oi, m0, t0, nthreads=8, want_m=False)
    for polish in (False, True):
        g = ctx.solve(inst, R, 0.0, 48.0, m0=m0, t0=t0, precision="fp8", polish=polish,
                      outputs=("energies", "spins"))
        assert np.array_equal(g.energies, O.energies(oi, g.spins))
        assert g.best_energy == O.energy(oi, g.best_spins)
        assert abs(g.best_energy - o["energy"].min()) <= 0.01 * abs(o["energy"].min())
    ctx.free(inst)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("n,R", [(512, 200), (640, 96)])
def test_paired_panel_gemm(ctx, monkeypatch, precision, n, R):
    """Panels 2q and 2q+1 share one GEMM: panel 2q over every K block, panel
    2q+1 over all but panel 2q's, whose new spins reach it in FP32 through
    chain 2q. With +-1 couplings only inside 256-spin blocks (pairs of panels)
    and start states exact in the operand format, one contracting sweep then
    equals the FP64 sweep to 1e-5 (n = 640 ends on an unpaired panel), for
    every replicas-per-warp choice alike."""
    J = block_diagonal_pm1(n, n + 1, block=256)
    inst = ctx.add_dense(J)
    m0 = (fp8_exact_m0 if precision == "fp8" else bf16_exact_m0)(R, n, 8)
    t0 = np.random.default_rng(9).uniform(110.0, 114.0, size=R).astype(np.float32)
    oi = O.Instance.dense(J)
    o = O.mars_solve(oi, m0, t0, c_step=60.0, fixed_sweeps=1)
    kw = dict(c_step=60.0, fixed_sweeps=1, m0=m0, t0=t0, precision=precision,
              outputs=("m_final", "energies", "spins"))
    monkeypatch.setenv("MARS_TC_PAIR", "1")
    runs = []
    for rpw in (1, 2, 4):
        monkeypatch.setenv("MARS_TC_RPW", str(rpw))
        runs.append(ctx.solve(inst, R, float(t0.min()), float(t0.max()), **kw))
    err = np.abs(runs[0].m_final - o["m"]).max()
    assert err <= 1e-5, err
    for r in runs[1:]:
        assert np.array_equal(r.m_final, runs[0].m_final)
    assert np.array_equal(runs[0].energies, O.energies(oi, runs[0].spins))
    ctx.free(inst)


def test_paired_panels_sk_quality(ctx, monkeypatch):
    n, R = 512, 256
    J = I.sk_pm1(n, 7)
    inst = ctx.add_dense(J)
    m0, t0 = I.replica_inputs(R, n, 0.0, 48.0, 8)
    oi = O.Instance.dense(J)
    o = O.mars_solve(oi, m0, t0, nthreads=8, want_m=False)
    monkeypatch.setenv("MARS_TC_PAIR", "1")
    for prec in ("bf16", "fp8"):
        g = ctx.solve(inst, R, 0.0, 48.0, m0=m0, t0=t0, precision=prec, outputs=("energies", "spins"))
        assert np.array_equal(g.energies, O.energies(oi, g.spins))
        assert abs(g.best_energy - o["energy"].min()) <= 0.01 * abs(o["energy"].min()), prec
    ctx.free(inst)


def test_persistent_sweeps_match_oracle(ctx, monkeypatch):
    """The opt-in persistent batches (one cooperative launch of chain and GEMM
    CTAs per batch of sweeps, MARS_TC_PERSIST=1): one contracting sweep over
    256-spin +-1 blocks with exact operands equals the FP64 sweep to 1e-5 (the
    chain feeds the next panel in FP32 across a block boundary), and a full
    SK solve returns exact energies."""
    monkeypatch.setenv("MARS_TC_PERSIST", "1")
    n, R = 1024, 200
    J = block_diagonal_pm1(n, n + 3, block=256)
    inst = ctx.add_dense(J)
    m0 = bf16_exact_m0(R, n, 8)
    t0 = np.random.default_rng(9).uniform(110.0, 114.0, size=R).astype(np.float32)
    oi = O.Instance.dense(J)
    o = O.mars_solve(oi, m0, t0, c_step=60.0, fixed_sweeps=1)
    g = ctx.solve(inst, R, float(t0.min()), float(t0.max()), c_step=60.0, fixed_sweeps=1, m0=m0, t0=t0,
                  precision="bf16", outputs=("m_final",))
    assert np.abs(g.m_final - o["m"]).max() <= 1e-5
    ctx.free(inst)
    J = I.sk_pm1(384, 12)
    inst = ctx.add_dense(J)
    g = ctx.solve(inst, 256, 0.0, 39.0, seed=3, precision="bf16", outputs=("energies", "spins", "sweeps"))
    oi = O.Instance.dense(J)
    assert np.array_equal(g.energies, O.energies(oi, g.spins))
    assert (g.replica_sweeps > 3).any()  # several sweeps, so several batches of the launch
    ctx.free(inst)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_chain_warps_do_not_change_results(ctx, monkeypatch, precision):
    """With few replicas active the plan runs each chain CTA with 4 warps
    instead of 8 (more CTAs, one warp per scheduler). A replica's chain is
    the same arithmetic either way: a whole solve under the paper's stopping
    rule returns identical spins, final magnetisations, energies and counts
    with 4 and with 8 chain warps forced."""
    n, R = 1024, 200
    J = I.sk_pm1(n, 41)
    inst = ctx.add_dense(J)
    m0, t0 = I.replica_inputs(R, n, 0.0, 8.0, 42)
    out = {}
    for cw in ("4", "8"):
        monkeypatch.setenv("MARS_TC_CHAIN_WARPS", cw)
        out[cw] = ctx.solve(inst, R, 0.0, 8.0, c_step=0.5, m0=m0, t0=t0, precision=precision,
                            outputs=("energies", "spins", "m_final", "sweeps", "levels", "capped"))
    a, b = out["4"], out["8"]
    assert np.array_equal(a.energies, b.energies) and np.array_equal(a.spins, b.spins)
    assert np.array_equal(a.m_final, b.m_final)
    assert np.array_equal(a.replica_sweeps, b.replica_sweeps)
    assert np.array_equal(a.replica_levels, b.replica_levels)
    assert np.array_equal(a.replica_capped, b.replica_capped)
    assert a.replica_sweeps.max() > a.replica_levels.max()
    ctx.free(inst)


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_compaction_does_not_change_results(ctx, monkeypatch, precision):
    """Between batches of sweeps the active replicas move to the first slots,
    so that the GEMM tiles and chain CTAs cover only them. Start temperatures
    spread over U(0, 8) with C_step 0.5 make replicas finish at different
    times; the whole solve with compaction equals the one without (spins,
    final magnetisations, energies and counts), and compaction did run (its
    two kernels per compaction add to the launch count)."""
    n, R = 1024, 300
    J = I.sk_pm1(n, 43)
    inst = ctx.add_dense(J)
    m0, t0 = I.replica_inputs(R, n, 0.0, 8.0, 44)
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("MARS_TC_COMPACT", flag)
        out[flag] = ctx.solve(inst, R, 0.0, 8.0, c_step=0.5, m0=m0, t0=t0, precision=precision,
                              outputs=("energies", "spins", "m_final", "sweeps", "levels", "capped"))
    a, b = out["1"], out["0"]
    assert np.array_equal(a.energies, b.energies) and np.array_equal(a.spins, b.spins)
    assert np.array_equal(a.m_final, b.m_final)
    assert np.array_equal(a.replica_sweeps, b.replica_sweeps)
    assert np.array_equal(a.replica_levels, b.replica_levels)
    assert np.array_equal(a.replica_capped, b.replica_capped)
    assert a.best_energy == b.best_energy and a.best_replica == b.best_replica
    assert a.kernel_launches > b.kernel_launches
    ctx.free(inst)


def test_compaction_skipped_when_its_scratch_does_not_fit(monkeypatch):
    """Compaction takes scratch only when it fits in the HBM budget: under the
    smallest budget a solve needs without it (found by bisection), the
    default solve still runs and returns the same results."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_05124_gb300 import build, mars
    from paper_1907_05124_gb300.mars import MarsError
    build.build()
    n, R = 1024, 300
    J = I.sk_pm1(n, 45)
    m0, t0 = I.replica_inputs(R, n, 0.0, 8.0, 46)

    def run(budget):
        c = mars.Context(0, hbm_budget_bytes=budget)
        try:
            inst = c.add_dense(J)
            return c.solve(inst, R, 0.0, 8.0, c_step=0.5, m0=m0, t0=t0, precision="bf16",
                           outputs=("energies", "sweeps"))
        except MarsError:
            return None
        finally:
            c.close()

    monkeypatch.setenv("MARS_TC_COMPACT", "0")
    lo, hi = 1 << 20, 8 << 30
    ref = run(hi)
    assert ref is not None
    while hi - lo > (1 << 20):
        mid = (lo + hi) // 2
        if run(mid) is not None:
            hi = mid
        else:
            lo = mid
    monkeypatch.setenv("MARS_TC_COMPACT", "1")
    got = run(hi)
    assert got is not None, "the default solve failed under the budget the solve itself needs"
    assert np.array_equal(got.energies, ref.energies)
    assert np.array_equal(got.replica_sweeps, ref.replica_sweeps)
