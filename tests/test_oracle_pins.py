"""Pins for the FP64 oracle, against things other than the oracle itself.

Each test ties one oracle function to a closed form, a library routine, an
invariant of the dynamics, brute force, or published generator values, so that
a dropped term, a wrong sign, a wrong update order or a transposed operand in
the oracle fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1907_05124_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Philox4x32-10 against published known-answer vectors
# --------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_draw_replicas_ranges_and_uniformity():
    from scipy import stats
    m0, t0 = O.draw_replicas(seed=12345, R=64, n=257, t_min=0.5, t_max=3.5)
    assert m0.dtype == np.float32 and t0.dtype == np.float32
    assert np.all(m0 >= -1.0) and np.all(m0 < 1.0)
    assert np.all(t0 >= 0.5) and np.all(t0 <= 3.5)
    # m0 is 2u-1 with u on a 2^-24 grid: (m0+1)/2 * 2^24 must be an integer.
    g = (m0.astype(np.float64) + 1.0) * 2.0 ** 23
    assert np.all(g == np.floor(g))
    assert stats.kstest(m0.ravel(), "uniform", args=(-1, 2)).pvalue > 1e-4
    assert stats.kstest(t0, "uniform", args=(0.5, 3.0)).pvalue > 1e-4
    # Counter-based: a sub-range of replicas is the same draw.
    m1, t1 = O.draw_replicas(seed=12345, R=8, n=257, t_min=0.5, t_max=3.5, r0=10)
    assert np.array_equal(m1, m0[10:18]) and np.array_equal(t1, t0[10:18])
    # Different streams and seeds give different draws.
    m2, _ = O.draw_replicas(seed=12345, R=4, n=257, t_min=0.5, t_max=3.5, stream=1)
    assert not np.array_equal(m2, m0[:4])


# --------------------------------------------------------------------------
# Exact summation against the library's correctly rounded sum
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["cancel", "ties", "random", "wide", "tiny"])
def test_exact_sum_matches_fsum(case):
    rng = np.random.default_rng(3)
    if case == "cancel":
        x = np.array([1e100, 1.0, -1e100, 3.5, 1e-30, -3.5])
    elif case == "ties":
        x = np.array([1.0, 2.0 ** -53, 2.0 ** -105, -2.0 ** -105])
    elif case == "random":
        x = rng.normal(size=20000) * np.exp(rng.uniform(-30, 30, size=20000))
    elif case == "wide":
        x = np.concatenate([rng.normal(size=500) * 1e300, rng.normal(size=500) * 1e-300,
                            -rng.normal(size=500) * 1e300])
    else:
        x = np.array([5e-324, 5e-324, 1e-310, -3e-320])
    assert O.exact_sum(x) == math.fsum(x.tolist())


def test_exact_sum_matches_fractions_small():
    rng = np.random.default_rng(4)
    for _ in range(50):
        x = rng.normal(size=7) * 10.0 ** rng.integers(-8, 8, size=7)
        exact = sum(Fraction(float(v)) for v in x)
        assert O.exact_sum(x) == float(exact)


# --------------------------------------------------------------------------
# Energy and cut (Eq. 2 with pairs once, Eq. 3)
# --------------------------------------------------------------------------

def test_energy_integer_couplings_exact():
    J = I.sk_pm1(97, 5)
    inst = O.Instance.dense(J)
    rng = np.random.default_rng(0)
    Ji = J.astype(np.int64)
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=97)
        si = s.astype(np.int64)
        pairs = int(np.triu(np.outer(si, si) * Ji, 1).sum())
        assert O.energy(inst, s) == pairs
        assert O.energy_quadratic(inst, s) == pairs


def test_energy_with_field_gaussian_against_fsum():
    n = 60
    J = I.sk_gauss(n, 2)
    h = np.random.default_rng(1).normal(size=n)
    inst = O.Instance.dense(J, h)
    s = np.random.default_rng(2).choice(np.array([-1, 1], dtype=np.int8), size=n)
    terms = [J[i, j] * s[i] * s[j] for i in range(n) for j in range(i + 1, n)]
    terms += [h[i] * s[i] for i in range(n)]
    assert O.energy(inst, s) == math.fsum(terms)
    assert O.energy_quadratic(inst, s) == pytest.approx(math.fsum(terms), rel=1e-12, abs=1e-12)


def test_energy_dense_and_csr_agree():
    csr = I.er_graph(300, 7, 3, "pm1")
    J = I.csr_to_dense(csr)
    s = np.random.default_rng(5).choice(np.array([-1, 1], dtype=np.int8), size=300)
    assert O.energy(O.Instance.csr(csr), s) == O.energy(O.Instance.dense(J), s)


def test_cut_direct_count_and_eq3_identity():
    csr = I.er_graph(200, 9, 4, "pm1")
    inst = O.Instance.csr(csr)
    rng = np.random.default_rng(6)
    row_ptr, col, val = csr
    rows = np.repeat(np.arange(200), np.diff(row_ptr))
    upper = col > rows
    W = val[upper].sum()
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], dtype=np.int8), size=200)
        direct = sum(v for i, j, v in zip(rows[upper], col[upper], val[upper]) if s[i] != s[j])
        assert O.cut(inst, s) == direct
        # Eq. 3 with the ordered-pair double sums: 1/4 sum J - 1/4 sum J s s.
        Jd = I.csr_to_dense(csr)
        eq3 = 0.25 * Jd.sum() - 0.25 * float(s.astype(float) @ Jd @ s.astype(float))
        assert O.cut(inst, s) == eq3
        assert O.cut(inst, s) == (W - O.energy(inst, s)) / 2


# --------------------------------------------------------------------------
# Brute force
# --------------------------------------------------------------------------

def _all_energies(J, h=None):
    n = J.shape[0]
    states = ((np.arange(2 ** n)[:, None] >> np.arange(n)) & 1) * 2 - 1
    S = states.astype(np.float64)
    e = 0.5 * np.einsum("ki,ij,kj->k", S, J, S)
    if h is not None:
        e += S @ h
    return e, states


def test_bruteforce_against_vectorised_enumeration():
    for seed in range(3):
        J = I.sk_pm1(11, seed)
        h = np.random.default_rng(seed).integers(-2, 3, size=11).astype(float)
        e_all, states = _all_energies(J, h)
        e, s, cnt = O.bruteforce(O.Instance.dense(J, h))
        assert e == e_all.min()
        assert cnt == int(np.sum(e_all == e_all.min()))
        assert O.energy(O.Instance.dense(J, h), s) == e


def test_bruteforce_ferromagnet_closed_form():
    n = 14
    J = -np.ones((n, n))
    np.fill_diagonal(J, 0)
    e, s, cnt = O.bruteforce(O.Instance.dense(J))
    assert e == -n * (n - 1) / 2 and cnt == 2 and abs(int(s.sum())) == n


def test_bruteforce_bipartite_antiferromagnet():
    csr = I.ea_lattice(4, 2, 0, "antiferro")  # 16 spins, 32 bonds, bipartite
    e, s, cnt = O.bruteforce(O.Instance.csr(csr))
    assert e == -32 and cnt == 2
    grid = s.reshape(4, 4).astype(int)
    assert np.all(grid * np.roll(grid, 1, 0) == -1) and np.all(grid * np.roll(grid, 1, 1) == -1)


# --------------------------------------------------------------------------
# Algorithm 1: closed forms and invariants
# --------------------------------------------------------------------------

def _levels_by_hand(t0, c):
    T, out = float(t0), []
    while True:
        T = T - c
        if not T > 0:
            return out
        out.append(T)


def test_temperature_levels_sequence():
    n = 8
    inst = O.Instance.dense(np.zeros((n, n)), np.linspace(-1, 1, n))
    t0 = np.array([0.0, 0.5, 1.0, 1.0000001, 3.25, 7.0], dtype=np.float32)
    m0 = np.zeros((len(t0), n), dtype=np.float32)
    r = O.mars_solve(inst, m0, t0, c_step=1.0)
    for k, t in enumerate(t0):
        lv = _levels_by_hand(float(t), 1.0)
        assert r["levels"][k] == len(lv)
        assert r["final_T"][k] == (lv[-1] if lv else 0.0)


def test_fields_only_closed_form():
    """J = 0: a level's first sweep lands on -tanh(h/T); the second has d = 0."""
    n = 16
    h = np.linspace(-2.0, 2.0, n)
    inst = O.Instance.dense(np.zeros((n, n)), h)
    m0, t0 = I.replica_inputs(6, n, 1.5, 6.0, 7)
    r = O.mars_solve(inst, m0, t0, c_step=1.0, d_min=1e-4)
    for k in range(6):
        lv = _levels_by_hand(float(t0[k]), 1.0)
        # numpy's tanh and the C library's may differ in the last bit
        np.testing.assert_allclose(r["m"][k], -np.tanh(h / lv[-1]), rtol=4e-16, atol=0)
        # each level: 2 sweeps unless the first already moved nothing beyond d_min
        assert r["sweeps"][k] == 2 * len(lv)
        assert r["capped_levels"][k] == 0


@pytest.mark.parametrize("k_max", [1, 2, 3, 7])
def test_k_max_cap_counts_on_fields_only_levels(k_max):
    """The cap on sweeps per level, against the fields-only closed form.

    With J = 0 a level's first sweep lands on -tanh(h/T) and its second moves
    nothing (d = 0). So k_max = 1 ends every level after one sweep with d > d_min
    (every level capped), while k_max >= 2 ends it on the second sweep with
    d = 0: a level that converges on exactly its k_max-th sweep is not capped."""
    n = 8
    h = np.linspace(0.5, 2.0, n)
    inst = O.Instance.dense(np.zeros((n, n)), h)
    t0 = np.array([3.5, 5.25], dtype=np.float32)
    m0 = np.zeros((2, n), dtype=np.float32)  # the first sweep moves every spin by tanh(h/T)
    r = O.mars_solve(inst, m0, t0, c_step=1.0, d_min=1e-4, k_max=k_max)
    for k in range(2):
        nl = len(_levels_by_hand(float(t0[k]), 1.0))
        if k_max == 1:
            assert r["sweeps"][k] == nl and r["capped_levels"][k] == nl
        else:
            assert r["sweeps"][k] == 2 * nl and r["capped_levels"][k] == 0


def _two_spin_jacobi_amplitudes(a0, J, Ts, k_max):
    """|s| after each synchronous sweep of the symmetric two-spin state."""
    a, out = a0, []
    for T in Ts:
        for _ in range(k_max):
            a = -math.tanh(J * a / T)
            out.append(abs(a))
    return out


@pytest.mark.parametrize("k_max", [1, 2, 5, 1000])
def test_k_max_cap_on_jacobi_two_cycle(k_max):
    """Synchronous sweeps of a two-spin antiferromagnet (J_12 = J > 0 in the
    paper's sign) below the stability bound T < J never converge.

    From s1 = s2 = a both spins stay equal and a <- -tanh(J a / T): the map
    flips the sign of a, and for J/T > 1 its second iterate has a non-zero
    attracting fixed point, so |a| never falls to 0 and every sweep moves each
    spin by |a_new| + |a_old| > d_min. Every level therefore takes exactly
    k_max sweeps and is counted as capped. Sequential sweeps of the same pair
    settle on the antiparallel fixed point instead and are never capped."""
    J = 4.0
    inst = O.Instance.dense(np.array([[0.0, J], [J, 0.0]]))
    t0 = np.array([3.5, 2.25], dtype=np.float32)   # levels 2.5, 1.5, 0.5 and 1.25, 0.25
    m0 = np.full((2, 2), 0.25, dtype=np.float32)
    r = O.mars_solve(inst, m0, t0, c_step=1.0, d_min=1e-4, k_max=k_max, update=O.UPDATE_JACOBI)
    for k in range(2):
        Ts = _levels_by_hand(float(t0[k]), 1.0)
        amps = _two_spin_jacobi_amplitudes(0.25, J, Ts, k_max)
        assert min(amps) > 1e-3  # the premise: the two-cycle never dies out
        assert r["levels"][k] == len(Ts)
        assert r["sweeps"][k] == k_max * len(Ts)
        assert r["capped_levels"][k] == len(Ts)
        # the state after the last sweep: both spins equal, of the amplitude by hand
        np.testing.assert_allclose(np.abs(r["m"][k]), amps[-1], rtol=1e-14, atol=0)
        assert r["m"][k][0] == r["m"][k][1]
    g = O.mars_solve(inst, m0, t0, c_step=1.0, d_min=1e-4, k_max=k_max, update=O.UPDATE_GS)
    if k_max >= 50:
        assert (g["capped_levels"] == 0).all()
        assert (g["m"][:, 0] * g["m"][:, 1] < 0).all()


def test_sweep_never_raises_mean_field_free_energy():
    """Sequential sweeps minimise the mean-field free energy one spin at a time.

    F(m) = sum_{i<j} J_ij m_i m_j + sum_i h_i m_i - T sum_i S(m_i), with S the
    binary entropy, is convex in each m_i and stationary at m_i = -tanh(Phi_i/T),
    so every GS sweep at fixed T must not increase F. A Jacobi sweep, a wrong
    sign or a dropped field breaks this.
    """
    def F(J, h, m, T):
        ent = -(((1 + m) / 2) * np.log((1 + m) / 2) + ((1 - m) / 2) * np.log((1 - m) / 2))
        return 0.5 * m @ J @ m + h @ m - T * ent.sum()

    n = 40
    J = I.sk_gauss(n, 9, sigma=1.0)
    h = np.random.default_rng(9).normal(size=n) * 0.3
    inst = O.Instance.dense(J, h)
    rng = np.random.default_rng(10)
    for T in (0.5, 2.0, 8.0):
        m = rng.uniform(-0.9, 0.9, size=n)
        f_prev = F(J, h, m, T)
        for _ in range(6):
            # one level at T: start at 2T and step by T
            r = O.mars_solve(inst, m[None].astype(np.float32), np.array([2 * T], np.float32),
                             c_step=T, fixed_sweeps=1)
            m = np.clip(r["m"][0], -1 + 1e-15, 1 - 1e-15)
            f = F(J, h, m, T)
            assert f <= f_prev + 1e-9 * (1 + abs(f_prev))
            f_prev = f
    # Jacobi on the same instance does raise F somewhere (the 2-cycle regime).
    m = rng.uniform(-0.9, 0.9, size=n)
    rises = 0
    f_prev = F(J, h, m, 0.5)
    for _ in range(10):
        r = O.mars_solve(inst, m[None].astype(np.float32), np.array([1.5], np.float32),
                         c_step=1.0, fixed_sweeps=1, update=O.UPDATE_JACOBI)
        m = np.clip(r["m"][0], -1 + 1e-15, 1 - 1e-15)
        f = F(J, h, m, 0.5)
        rises += f > f_prev + 1e-9
        f_prev = f
    assert rises > 0


def test_high_temperature_contraction():
    """T > ||J||_inf: one sweep shrinks max|m| by at least ||J||_inf / T."""
    csr = I.er_graph(150, 6, 11, "pm1")
    inst = O.Instance.csr(csr)
    J = I.csr_to_dense(csr)
    jinf = np.abs(J).sum(axis=1).max()
    T = 1.5 * jinf
    m0, _ = I.replica_inputs(5, 150, 0, 1, 12)
    for update in (O.UPDATE_GS, O.UPDATE_JACOBI):
        r = O.mars_solve(inst, m0, np.full(5, 2 * T, np.float32), c_step=T, fixed_sweeps=1,
                         update=update)
        for k in range(5):
            assert np.abs(r["m"][k]).max() <= (jinf / T) * np.abs(m0[k]).max() + 1e-15


def test_converged_state_is_a_fixed_point():
    """A level that stopped on d <= d_min leaves m within d_min*||J||_inf/T of the fixed point."""
    csr = I.ea_lattice(12, 2, 1)
    inst = O.Instance.csr(csr)
    J = I.csr_to_dense(csr)
    jinf = np.abs(J).sum(axis=1).max()
    m0, t0 = I.replica_inputs(8, csr.n, 0.0, 4.0, 13)
    r = O.mars_solve(inst, m0, t0, c_step=1.0, d_min=1e-4, k_max=5000)
    checked = 0
    for k in range(8):
        if r["levels"][k] == 0 or r["last_d"][k] > 1e-4:
            continue
        T = r["final_T"][k]
        m = r["m"][k]
        resid = np.abs(m + np.tanh(J @ m / T)).max()
        assert resid <= 1e-4 * jinf / T + 1e-12
        checked += 1
    assert checked >= 4


def test_gs_sweep_matches_sequential_definition_on_two_spins():
    """Two coupled spins: the second update of a GS sweep sees the first's new value."""
    a, h0, h1, T = 0.8, 0.3, -0.2, 0.75  # T + 1 exact in float32
    J = np.array([[0.0, a], [a, 0.0]])
    inst = O.Instance.dense(J, np.array([h0, h1]))
    s0, s1 = 0.4, -0.6
    r = O.mars_solve(inst, np.array([[s0, s1]], np.float32), np.array([T + 1], np.float32),
                     fixed_sweeps=1)
    s0f, s1f = np.float32(s0).item(), np.float32(s1).item()
    n0 = -math.tanh((a * s1f + h0) / T)
    n1 = -math.tanh((a * n0 + h1) / T)
    assert r["m"][0][0] == n0 and r["m"][0][1] == n1
    # in the reverse order the roles swap
    r = O.mars_solve(inst, np.array([[s0, s1]], np.float32), np.array([T + 1], np.float32),
                     fixed_sweeps=1, order=[1, 0])
    m1 = -math.tanh((a * s0f + h1) / T)
    m0 = -math.tanh((a * m1 + h0) / T)
    assert r["m"][0][0] == m0 and r["m"][0][1] == m1


def test_colour_order_sweep_equals_two_half_sweeps():
    """On a bipartite lattice a sweep in colour order is: all of colour 0 from the
    old colour-1 values, then all of colour 1 from the new colour-0 values."""
    csr = I.ea_lattice(6, 2, 2)
    J = I.csr_to_dense(csr)
    inst = O.Instance.csr(csr)
    order = I.greedy_colour_order(csr)
    colour0 = order[: csr.n // 2]
    colour1 = order[csr.n // 2:]
    assert np.all(J[np.ix_(colour0, colour0)] == 0) and np.all(J[np.ix_(colour1, colour1)] == 0)
    m0, _ = I.replica_inputs(1, csr.n, 0, 1, 3)
    T = 1.25
    r = O.mars_solve(inst, m0, np.array([2 * T], np.float32), c_step=T, fixed_sweeps=1,
                     order=order)
    m = m0[0].astype(np.float64).copy()
    m[colour0] = -np.tanh(J[colour0] @ m / T)
    m[colour1] = -np.tanh(J[colour1] @ m / T)
    np.testing.assert_allclose(r["m"][0], m, rtol=0, atol=1e-15)


def test_mars_never_beats_ground_state_and_finds_it_n20():
    """SK +-1, N = 20: every replica's energy is >= the brute-force ground state,
    and 256 replicas from T0 ~ U(0, 16) reach it."""
    J = I.sk_pm1(20, 0)
    inst = O.Instance.dense(J)
    e_gs, _, _ = O.bruteforce(inst)
    m0, t0 = I.replica_inputs(256, 20, 0.0, 16.0, 0)
    r = O.mars_solve(inst, m0, t0)
    assert np.all(r["energy"] >= e_gs)
    assert r["energy"].min() == e_gs
    for k in range(0, 256, 37):
        assert O.energy(inst, r["sigma"][k]) == r["energy"][k]


def test_ferromagnet_descent_aligns():
    n = 32
    J = -np.ones((n, n))
    np.fill_diagonal(J, 0)
    m0, t0 = I.replica_inputs(16, n, 0.0, 40.0, 1)
    r = O.mars_solve(O.Instance.dense(J), m0, t0)
    ok = r["levels"] > 0
    assert np.all(r["energy"][ok] == -n * (n - 1) / 2)


def test_antiferromagnet_lattice_reaches_checkerboard():
    csr = I.ea_lattice(8, 2, 0, "antiferro")
    m0, t0 = I.replica_inputs(32, csr.n, 0.0, 4.0, 2)
    r = O.mars_solve(O.Instance.csr(csr), m0, t0, order=I.greedy_colour_order(csr))
    assert r["energy"].min() == -csr.nnz // 2


# --------------------------------------------------------------------------
# cooling-schedule variants (labelled, not the paper's): geometric, quench
# --------------------------------------------------------------------------

def test_geometric_levels_closed_form():
    """Fields only, geometric cooling T <- r T while T > t_floor: the levels
    are t0 r, t0 r^2, ... down to the last one above t_floor, each landing on
    -tanh(h / T) in exactly two sweeps."""
    n = 40
    h = np.linspace(-1.5, 1.9, n)
    inst = O.Instance.dense(np.zeros((n, n)), h)
    r, floor_ = 0.75, 0.2
    t0 = np.array([3.0, 0.9, 0.25, 0.2], dtype=np.float32)
    m0 = np.zeros((t0.size, n), dtype=np.float32)
    out = O.mars_solve(inst, m0, t0, geometric=r, t_floor=floor_)
    for k, t in enumerate(t0.astype(np.float64)):
        levels, T = 0, t
        while T * r > floor_:
            T *= r
            levels += 1
        assert out["levels"][k] == levels
        assert out["sweeps"][k] == 2 * levels
        if levels:
            assert out["final_T"][k] == T
            np.testing.assert_allclose(out["m"][k], -np.tanh(h / T), rtol=4e-16, atol=1e-300)
        else:
            assert np.all(out["m"][k] == 0.0)


def test_quench_fields_only_closed_form():
    """The quench level takes the update's T -> 0+ limit, s_i = -sgn(Phi_i):
    with fields only it lands on -sgn(h) in one sweep and stops after the
    second (no change); a zero field gives 0."""
    h = np.array([-2.0, -1e-9, 0.0, 3e-12, 0.5, 7.0])
    n = h.size
    inst = O.Instance.dense(np.zeros((n, n)), h)
    m0 = np.random.default_rng(1).uniform(-1, 1, size=(2, n)).astype(np.float32)
    t0 = np.array([0.5, 2.5], dtype=np.float32)  # no level, then two linear levels
    out = O.mars_solve(inst, m0, t0, quench=True)
    assert np.array_equal(out["m"][0], -np.sign(h))
    assert np.array_equal(out["m"][1], -np.sign(h))
    assert list(out["levels"]) == [1, 3]
    assert list(out["sweeps"]) == [2, 2 * 2 + 2]
    assert list(out["final_T"]) == [0.0, 0.0]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_quench_ends_in_single_flip_local_minimum(seed):
    """After the quench level converges every spin sits against its field, so
    no single flip lowers the exact energy (E changes by -2 sigma_i Phi_i >= 0
    under a flip of i). With N = 40 (+-1 couplings) every field of a +-1
    state is an odd integer, never 0."""
    n = 40
    J = I.sk_pm1(n, seed)
    inst = O.Instance.dense(J)
    m0, t0 = I.replica_inputs(16, n, 0.0, 12.0, seed + 10)
    out = O.mars_solve(inst, m0, t0, quench=True)
    for r in range(16):
        m = out["m"][r]
        assert np.all(np.abs(m) == 1.0), m  # converged onto +-1 spins
        sig = out["sigma"][r]
        e = O.energy(inst, sig)
        for i in range(n):
            flip = sig.copy()
            flip[i] = -flip[i]
            assert O.energy(inst, flip) >= e


# --------------------------------------------------------------------------
# Noisy mean-field annealing (Section 2): the alternative epilogue
# --------------------------------------------------------------------------

def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            v = [int(x, 16) for x in ln.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_nmfa_normal_box_muller_of_published_philox_words():
    """The noise is the Box-Muller transform of the first two words of
    Philox at counter (i/2, r, 2 + k, stream) under key (seed): choose the
    arguments so that counter and key are a published known-answer vector."""
    for ctr, key, out in _kat_rows():
        i0 = 2 * ctr[0]
        if i0 >= 2**32:
            continue  # the spin index is 32-bit: this counter word is out of reach
        seed = key[0] | (key[1] << 32)
        k = (ctr[2] - 2) % 2**32
        u1 = ((out[0] >> 8) + 1) * 2.0**-24
        u2 = (out[1] >> 8) * 2.0**-24
        rho = math.sqrt(-2.0 * math.log(u1))
        assert O.nmfa_normal(seed, ctr[3], ctr[1], k, i0) == pytest.approx(
            rho * math.cos(2 * math.pi * u2), rel=1e-15, abs=1e-15)
        assert O.nmfa_normal(seed, ctr[3], ctr[1], k, i0 + 1) == pytest.approx(
            rho * math.sin(2 * math.pi * u2), rel=1e-15, abs=1e-15)


def test_nmfa_normal_is_standard_normal():
    from scipy import stats
    x = np.array([O.nmfa_normal(7, 1, r, k, i) for r in range(5) for k in range(40) for i in range(500)])
    assert abs(x.mean()) < 4.0 / math.sqrt(len(x))
    assert abs(x.var() - 1.0) < 0.03
    assert stats.kstest(x, "norm").pvalue > 1e-3
    # the two normals of one Box-Muller pair are uncorrelated
    ev = np.array([O.nmfa_normal(3, 0, 0, 0, 2 * q) for q in range(20000)])
    od = np.array([O.nmfa_normal(3, 0, 0, 0, 2 * q + 1) for q in range(20000)])
    assert abs(np.corrcoef(ev, od)[0, 1]) < 0.03


def test_nmfa_zero_mixing_moves_nothing():
    J = I.sk_pm1(24, 3)
    m0, t0 = I.replica_inputs(4, 24, 2.0, 9.0, 4)
    r = O.nmfa_solve(O.Instance.dense(J), m0, t0, alpha=0.0, sigma=0.7, seed=5)
    assert np.array_equal(r["m"], m0.astype(np.float64))


def test_nmfa_fields_only_closed_form_with_mixing():
    """J = 0: the normalised field is h_i / |h_i| = sign(h_i), so each
    iteration at T_k sets s <- alpha (-tanh(sign(h)/T_k)) + (1 - alpha) s."""
    n = 6
    h = np.array([0.3, -2.0, 5.0, -0.01, 1.0, 0.0])
    inst = O.Instance.dense(np.zeros((n, n)), h)
    m0 = np.linspace(-0.9, 0.8, n).astype(np.float32)[None, :]
    t0 = np.array([3.75], dtype=np.float32)
    a = 0.3
    r = O.nmfa_solve(inst, m0, t0, c_step=1.0, alpha=a, sigma=0.0)
    s = m0[0].astype(np.float64)
    for T in (2.75, 1.75, 0.75):
        s = a * (-np.tanh(np.sign(h) / T)) + (1 - a) * s
    np.testing.assert_allclose(r["m"][0], s, rtol=0, atol=1e-15)
    assert r["levels"][0] == 3 and r["sweeps"][0] == 3 and r["capped_levels"][0] == 0


def test_nmfa_field_is_normalised():
    """Scaling J and h by a > 0 leaves every normalised field, and therefore
    the whole trajectory, unchanged (noise included)."""
    J = I.sk_gauss(40, 2)
    h = np.random.default_rng(3).normal(size=40)
    m0, t0 = I.replica_inputs(3, 40, 0.5, 3.0, 9)
    kw = dict(c_step=0.25, alpha=0.6, sigma=0.2, seed=11)
    a = O.nmfa_solve(O.Instance.dense(J, h), m0, t0, **kw)
    b = O.nmfa_solve(O.Instance.dense(37.5 * J, 37.5 * h), m0, t0, **kw)
    np.testing.assert_allclose(a["m"], b["m"], rtol=0, atol=1e-12)
    assert np.abs(a["m"] - m0).max() > 0.1  # the trajectory did move


def test_nmfa_without_noise_is_synchronous_mars_on_regular_rows():
    """With sigma = 0 and alpha = 1, on an instance whose rows all have the
    same norm c (h = 0, +-1 couplings, every spin of the same degree), an
    iteration at T is a synchronous MARS sweep at temperature c T; one
    iteration per level. So NMFA(t0, C_step) equals the oracle's synchronous
    MARS with one sweep per level from c t0 in steps of c C_step."""
    csr = I.ea_lattice(6, 2, 1)  # degree 4: c = 2
    inst = O.Instance.csr(csr)
    m0, t0 = I.replica_inputs(4, csr.n, 1.0, 3.0, 2)
    a = O.nmfa_solve(inst, m0, t0, c_step=0.5, alpha=1.0, sigma=0.0)
    b = O.mars_solve(inst, m0, (2.0 * t0).astype(np.float32), c_step=1.0, fixed_sweeps=1,
                     update=O.UPDATE_JACOBI)
    np.testing.assert_allclose(a["m"], b["m"], rtol=0, atol=1e-12)
    assert np.array_equal(a["levels"], b["levels"]) and np.array_equal(a["sweeps"], b["levels"])


def test_nmfa_noise_enters_with_scale_sigma():
    """J = 0, h = 0, alpha = 1: one iteration gives s_i = -tanh(sigma xi_i / T),
    so T atanh(-s_i) / sigma over many spins is standard normal."""
    from scipy import stats
    n = 4000
    inst = O.Instance.csr((np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0)))
    m0 = np.zeros((2, n), dtype=np.float32)
    t0 = np.array([1.5, 1.5], dtype=np.float32)  # one level at T = 0.5
    r = O.nmfa_solve(inst, m0, t0, c_step=1.0, alpha=1.0, sigma=0.3, seed=4)
    z = (0.5 * np.arctanh(-r["m"]) / 0.3).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert not np.array_equal(r["m"][0], r["m"][1])  # each replica draws its own noise
    # the last iteration's noise alone decides s, and a new iteration draws anew
    t2 = np.array([2.5, 2.5], dtype=np.float32)  # levels at T = 1.5, then 0.5
    r2 = O.nmfa_solve(inst, m0, t2, c_step=1.0, alpha=1.0, sigma=0.3, seed=4)
    z2 = (0.5 * np.arctanh(-r2["m"]) / 0.3).ravel()
    assert stats.kstest(z2, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.06


def test_time_to_target_golden_is_the_oracles_own():
    """The stored time-to-target energy of the dense SK instance N = 1024 is
    what the oracle returns for the stored best replica: re-running that one
    replica (its start state from the oracle's draw, seed 0) reproduces the
    energy exactly, and no replica is stored as better than that."""
    import json
    import os
    from paper_1907_05124_gb300 import instances
    path = os.path.join(os.path.dirname(__file__), "golden", "sk_gauss1024_target.json")
    rec = json.load(open(path))
    r = rec["best_replica"]
    m0, t0 = O.draw_replicas(0, r + 1, 1024, 0.0, 2.0)
    assert float(t0[r]) == rec["best_replica_t0"]
    oi = O.Instance.dense(instances.sk_gauss(1024, 3))
    o = O.mars_solve(oi, m0[r:r + 1], t0[r:r + 1], c_step=1.0 / np.sqrt(1024), d_min=1e-4, k_max=1000,
                     want_m=False)
    assert float(o["energy"][0]) == rec["best_energy"]
    assert rec["hits"] >= 1 and rec["energy_p10"] >= rec["best_energy"]
