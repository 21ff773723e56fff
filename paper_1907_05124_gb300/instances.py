"""Seeded synthetic problem instances and replica inputs.

This module only draws inputs: coupling matrices, fields, sweep orders and
random start states. It holds none of the annealing arithmetic, so both the
CUDA library's tests and the CPU oracle's tests may draw from it.

Instance families follow the problem statement of the paper (Section 2):

* Sherrington-Kirkpatrick (SK): every pair coupled, ``J`` symmetric with a zero
  diagonal, entries either uniform in {-1, +1} or Gaussian.
* Edwards-Anderson (EA): nearest-neighbour +-J couplings on a periodic
  square (2-D) or cubic (3-D) lattice.
* Erdos-Renyi graphs with weights {+1} or {-1, +1}, the max-cut workloads
  shaped like the random G-set rows the paper evaluates (Section 4.3).

Sparse instances are CSR triplets ``(row_ptr int32[n+1], col int32[nnz],
val float64[nnz])`` holding both directions of every edge (the matrix is
symmetric) with columns sorted within each row. Dense instances are
``float64[n, n]`` arrays.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "sk_pm1",
    "sk_gauss",
    "ea_lattice",
    "er_graph",
    "dense_to_csr",
    "csr_to_dense",
    "greedy_colour_order",
    "replica_inputs",
    "Csr",
]


class Csr(tuple):
    """A ``(row_ptr, col, val)`` triple with a few read-only conveniences."""

    __slots__ = ()

    def __new__(cls, row_ptr, col, val):
        return super().__new__(cls, (np.ascontiguousarray(row_ptr, dtype=np.int32),
                                     np.ascontiguousarray(col, dtype=np.int32),
                                     np.ascontiguousarray(val, dtype=np.float64)))

    @property
    def row_ptr(self):
        return self[0]

    @property
    def col(self):
        return self[1]

    @property
    def val(self):
        return self[2]

    @property
    def n(self) -> int:
        return int(self[0].shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self[1].shape[0])


def _symmetric_from_upper(upper: np.ndarray) -> np.ndarray:
    u = np.triu(upper, 1)
    return u + u.T


def sk_pm1(n: int, seed: int) -> np.ndarray:
    """Dense SK instance with J_ij uniform in {-1, +1} (i<j), mirrored, zero diagonal."""
    rng = np.random.default_rng(seed)
    upper = rng.choice(np.array([-1.0, 1.0]), size=(n, n))
    return _symmetric_from_upper(upper)


def sk_gauss(n: int, seed: int, sigma: float | None = None) -> np.ndarray:
    """Dense SK instance with J_ij ~ Normal(0, sigma^2) (default sigma = 1/sqrt(n))."""
    rng = np.random.default_rng(seed)
    s = 1.0 / np.sqrt(n) if sigma is None else float(sigma)
    upper = rng.normal(0.0, s, size=(n, n))
    return _symmetric_from_upper(upper)


def sk_uniform(n: int, seed: int) -> np.ndarray:
    """Dense SK instance with J_ij uniform in (-1, 1) (i<j), mirrored, zero
    diagonal: the coupling scale (standard deviation 1/sqrt(3)) that the
    paper's printed SK energies and temperature windows correspond to."""
    rng = np.random.default_rng(seed)
    upper = rng.uniform(-1.0, 1.0, size=(n, n))
    return _symmetric_from_upper(upper)


def _csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray) -> Csr:
    """Symmetric CSR from an undirected edge list (each edge listed once)."""
    rows = np.concatenate([src, dst]).astype(np.int64)
    cols = np.concatenate([dst, src]).astype(np.int64)
    vals = np.concatenate([w, w]).astype(np.float64)
    key = rows * n + cols
    perm = np.argsort(key, kind="stable")
    rows, cols, vals, key = rows[perm], cols[perm], vals[perm], key[perm]
    if key.size and np.any(key[1:] == key[:-1]):
        raise ValueError("duplicate edge in edge list")
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Csr(row_ptr, cols, vals)


def ea_lattice(L: int, dim: int, seed: int, weights: str = "pm1") -> Csr:
    """Periodic EA lattice of side L in 2 or 3 dimensions.

    Every site bonds to its +1 neighbour along each axis (periodic), so the
    lattice has ``dim * L**dim`` bonds and every site has ``2*dim`` neighbours.
    ``weights`` is ``"pm1"`` (uniform in {-1, +1}), ``"ferro"`` (all -1, the
    aligned ground state in the paper's sign) or ``"antiferro"`` (all +1).
    """
    if dim not in (2, 3):
        raise ValueError("dim must be 2 or 3")
    if L < 3:
        raise ValueError("L must be >= 3 so that periodic bonds are distinct")
    rng = np.random.default_rng(seed)
    shape = (L,) * dim
    n = L ** dim
    idx = np.arange(n).reshape(shape)
    src, dst, w = [], [], []
    for axis in range(dim):
        nb = np.roll(idx, -1, axis=axis)
        src.append(idx.ravel())
        dst.append(nb.ravel())
        if weights == "pm1":
            w.append(rng.choice(np.array([-1.0, 1.0]), size=n))
        elif weights == "ferro":
            w.append(-np.ones(n))
        elif weights == "antiferro":
            w.append(np.ones(n))
        else:
            raise ValueError(weights)
    return _csr_from_edges(n, np.concatenate(src), np.concatenate(dst), np.concatenate(w))


def er_graph(n: int, mean_degree: float, seed: int, weights: str = "pm1") -> Csr:
    """Erdos-Renyi G(n, p) with p = mean_degree/(n-1); weights "one" or "pm1".

    The edge count is drawn from Binomial(n(n-1)/2, p) and that many distinct
    unordered pairs are then drawn uniformly, which is the G(n, p) law.
    """
    rng = np.random.default_rng(seed)
    p = float(mean_degree) / (n - 1)
    m = int(rng.binomial(n * (n - 1) // 2, p))
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        a = rng.integers(0, n, size=2 * (m - keys.size) + 16)
        b = rng.integers(0, n, size=a.size)
        keep = a != b
        lo, hi = np.minimum(a, b)[keep], np.maximum(a, b)[keep]
        keys = np.unique(np.concatenate([keys, lo * n + hi]))
    keys = rng.permutation(keys)[:m]
    i, j = keys // n, keys % n
    if weights == "one":
        w = np.ones(m)
    elif weights == "pm1":
        w = rng.choice(np.array([-1.0, 1.0]), size=m)
    else:
        raise ValueError(weights)
    return _csr_from_edges(n, i, j, w)


def dense_to_csr(J: np.ndarray) -> Csr:
    """CSR of the non-zero off-diagonal entries of a dense matrix."""
    J = np.asarray(J, dtype=np.float64)
    n = J.shape[0]
    mask = J != 0
    np.fill_diagonal(mask, False)
    rows, cols = np.nonzero(mask)
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Csr(row_ptr, cols, J[rows, cols])


def csr_to_dense(csr: Csr) -> np.ndarray:
    row_ptr, col, val = csr
    n = row_ptr.shape[0] - 1
    J = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    J[rows, col] = val
    return J


def greedy_colour_order(csr: Csr) -> np.ndarray:
    """A spin visiting order that lists greedy colour classes one after another.

    Vertices are coloured in index order with the smallest colour unused by
    their already coloured neighbours; the order lists colour 0's vertices in
    index order, then colour 1's, and so on. Within one colour class no two
    spins are coupled, which is what lets a sequential sweep in this order run
    one colour class at a time.
    """
    row_ptr, col, _ = csr
    n = row_ptr.shape[0] - 1
    colour = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        nb = col[row_ptr[i]:row_ptr[i + 1]]
        used = set(colour[nb][colour[nb] >= 0].tolist())
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return np.lexsort((np.arange(n), colour)).astype(np.int32)


def replica_inputs(R: int, n: int, t_min: float, t_max: float, seed: int):
    """Random start states for R replicas: m0 ~ U(-1, 1) and T0 ~ U(t_min, t_max).

    Both are returned as float32 (m0 of shape (R, n), replica-major, and T0 of
    shape (R,)), the values the library and the oracle both consume.
    """
    rng = np.random.default_rng(seed)
    m0 = rng.uniform(-1.0, 1.0, size=(R, n)).astype(np.float32)
    t0 = rng.uniform(t_min, t_max, size=R).astype(np.float32)
    return m0, t0
