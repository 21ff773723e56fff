"""The seeded input generators against the input recipe they implement.

These generators feed both the CUDA path's tests and the oracle's, so each
structural claim is checked here on the host: symmetry and a zero diagonal
(the problem statement of Section 2 needs both), the lattices' degree and
periodic neighbours, the coupling distributions, the Erdos-Renyi edge count,
the colour order's independent classes and the replica inputs' ranges.
"""
import numpy as np
import pytest

from paper_1907_05124_gb300 import instances as I


def _rows(csr):
    return np.repeat(np.arange(csr.n), np.diff(csr.row_ptr))


def _assert_symmetric_csr(csr):
    J = I.csr_to_dense(csr)
    assert np.array_equal(J, J.T)
    assert np.all(np.diag(J) == 0)
    # columns sorted and unique within each row
    for i in range(csr.n):
        c = csr.col[csr.row_ptr[i]:csr.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


@pytest.mark.parametrize("L,dim", [(5, 2), (6, 2), (4, 3)])
def test_ea_lattice_structure(L, dim):
    csr = I.ea_lattice(L, dim, 3)
    n = L ** dim
    assert csr.n == n and csr.nnz == 2 * dim * n
    assert np.all(np.diff(csr.row_ptr) == 2 * dim)
    assert set(np.unique(csr.val)) <= {-1.0, 1.0}
    _assert_symmetric_csr(csr)
    # site 0's neighbours are the periodic +-1 steps along each axis
    expect = set()
    for axis in range(dim):
        stride = L ** (dim - 1 - axis)
        expect |= {stride, (L - 1) * stride}
    assert set(csr.col[csr.row_ptr[0]:csr.row_ptr[1]].tolist()) == expect


def test_ea_lattice_sign_families():
    assert np.all(I.ea_lattice(4, 2, 0, "ferro").val == -1.0)
    assert np.all(I.ea_lattice(4, 2, 0, "antiferro").val == 1.0)
    v = I.ea_lattice(40, 2, 1).val
    assert abs(np.mean(v)) < 0.05  # +-1 equally likely: 3200 bonds, sd of the mean 0.018


@pytest.mark.parametrize("weights", ["one", "pm1"])
def test_er_graph_structure_and_edge_count(weights):
    n, d = 3000, 6.0
    csr = I.er_graph(n, d, 5, weights)
    _assert_symmetric_csr(csr)
    m = csr.nnz // 2
    mean = d * n / 2  # Binomial(n(n-1)/2, d/(n-1))
    assert abs(m - mean) < 5 * np.sqrt(mean)
    vals = set(np.unique(csr.val))
    assert vals == ({1.0} if weights == "one" else {-1.0, 1.0})


def test_sk_pm1_and_gaussian_and_uniform():
    n = 400
    A = I.sk_pm1(n, 0)
    assert np.array_equal(A, A.T) and np.all(np.diag(A) == 0)
    off = A[np.triu_indices(n, 1)]
    assert set(np.unique(off)) == {-1.0, 1.0}
    G = I.sk_gauss(n, 1)
    assert np.array_equal(G, G.T) and np.all(np.diag(G) == 0)
    g = G[np.triu_indices(n, 1)]
    assert abs(g.var() * n - 1.0) < 0.05  # variance 1/n; 79800 samples
    assert abs(g.mean()) < 5 * np.sqrt(1.0 / n / g.size)
    U = I.sk_uniform(n, 2)
    assert np.array_equal(U, U.T) and np.all(np.diag(U) == 0)
    u = U[np.triu_indices(n, 1)]
    assert u.min() > -1.0 and u.max() < 1.0
    assert abs(u.var() - 1.0 / 3.0) < 0.01


def test_dense_csr_round_trip():
    J = I.sk_gauss(50, 4)
    J[np.abs(J) < 0.05] = 0.0
    J = np.triu(J, 1)
    J = J + J.T
    csr = I.dense_to_csr(J)
    assert np.array_equal(I.csr_to_dense(csr), J)
    assert csr.nnz == np.count_nonzero(J)


@pytest.mark.parametrize("make", [lambda: I.ea_lattice(6, 2, 0), lambda: I.ea_lattice(4, 3, 0),
                                  lambda: I.er_graph(500, 7, 2, "pm1")])
def test_greedy_colour_order_lists_independent_classes(make):
    csr = make()
    order = I.greedy_colour_order(csr)
    assert np.array_equal(np.sort(order), np.arange(csr.n))
    # recompute the greedy colours and check the order's classes
    colour = np.full(csr.n, -1)
    for i in range(csr.n):
        nb = csr.col[csr.row_ptr[i]:csr.row_ptr[i + 1]]
        used = set(colour[nb][colour[nb] >= 0].tolist())
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    assert np.all(np.diff(colour[order]) >= 0)  # classes one after another
    rows = _rows(csr)
    assert np.all(colour[rows] != colour[csr.col])  # no edge inside a class


def test_even_lattice_takes_two_colours():
    order = I.greedy_colour_order(I.ea_lattice(6, 2, 0))
    first = order[:18]
    assert np.array_equal(np.sort(first), np.sort([i * 6 + j for i in range(6) for j in range(6)
                                                    if (i + j) % 2 == 0]))


def test_replica_inputs_ranges():
    m0, t0 = I.replica_inputs(64, 100, 0.5, 2.5, 9)
    assert m0.shape == (64, 100) and m0.dtype == np.float32
    assert t0.shape == (64,) and t0.dtype == np.float32
    assert m0.min() >= -1.0 and m0.max() <= 1.0
    assert t0.min() >= 0.5 and t0.max() <= 2.5
    m1, t1 = I.replica_inputs(64, 100, 0.5, 2.5, 9)
    assert np.array_equal(m0, m1) and np.array_equal(t0, t1)  # seeded
