"""MARS oracle: plain FP64 CPU restatement of the paper's method.

TEST INFRASTRUCTURE ONLY. The product library never imports this package;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` do. It shares no code with the CUDA path.

This module compiles ``mars_oracle.c`` with the system C compiler (in-tree,
into ``oracle/_lib``) and exposes it through ``ctypes``. See the header
``mars_oracle.h`` for the definitions each function restates (Section 2,
Eq. 2 and Eq. 3; Section 3, Algorithm 1).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, brute force, library routines, published Philox values).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mars_oracle.c")
_HDR = os.path.join(_HERE, "mars_oracle.h")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libmars_oracle.so")

UPDATE_GS = 0
UPDATE_JACOBI = 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    tmp = _LIB + f".tmp{os.getpid()}"
    base = [cc, "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:-3] + ["-fopenmp"] + base[-3:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Inst(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("J", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("h", ctypes.c_void_p)]


class ReplicaStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("levels", ctypes.c_int64),
                ("capped_levels", ctypes.c_int64), ("final_T", ctypes.c_double),
                ("last_d", ctypes.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.or_energy.restype = ctypes.c_double
        _lib.or_energy.argtypes = [P, P]
        _lib.or_energy_quadratic.restype = ctypes.c_double
        _lib.or_energy_quadratic.argtypes = [P, P]
        _lib.or_cut.restype = ctypes.c_double
        _lib.or_cut.argtypes = [P, P]
        _lib.or_exact_sum.restype = ctypes.c_double
        _lib.or_exact_sum.argtypes = [P, ctypes.c_int64]
        _lib.or_local_field.restype = ctypes.c_double
        _lib.or_local_field.argtypes = [P, P, ctypes.c_int32]
        _lib.or_bruteforce.restype = ctypes.c_int
        _lib.or_bruteforce.argtypes = [P, ctypes.c_double, P, P, P]
        _lib.or_mars_solve.restype = ctypes.c_int
        _lib.or_mars_solve.argtypes = [P, P, ctypes.c_int32, P, P, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, P, ctypes.c_int32, P, P, P, P]
        _lib.or_nmfa_normal.restype = ctypes.c_double
        _lib.or_nmfa_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32]
        _lib.or_nmfa_solve.restype = ctypes.c_int
        _lib.or_nmfa_solve.argtypes = [P, ctypes.c_int32, P, P, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32, P,
                                       ctypes.c_int32, P, P, P, P]
        _lib.or_philox4x32_10.restype = None
        _lib.or_philox4x32_10.argtypes = [P, P, P]
        _lib.or_draw_replicas.restype = None
        _lib.or_draw_replicas.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, P, P]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


@dataclass
class Instance:
    """Couplings for the oracle: a dense ``J`` or a CSR triple, plus optional ``h``."""

    n: int
    J: np.ndarray | None = None
    row_ptr: np.ndarray | None = None
    col: np.ndarray | None = None
    val: np.ndarray | None = None
    h: np.ndarray | None = None

    @classmethod
    def dense(cls, J, h=None):
        J = np.ascontiguousarray(J, dtype=np.float64)
        return cls(n=J.shape[0], J=J, h=None if h is None else np.ascontiguousarray(h, np.float64))

    @classmethod
    def csr(cls, csr, h=None):
        row_ptr, col, val = csr
        return cls(n=len(row_ptr) - 1, row_ptr=np.ascontiguousarray(row_ptr, np.int32),
                   col=np.ascontiguousarray(col, np.int32),
                   val=np.ascontiguousarray(val, np.float64),
                   h=None if h is None else np.ascontiguousarray(h, np.float64))

    def _c(self):
        s = _Inst(self.n, _ptr(self.J), _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val),
                  _ptr(self.h))
        return s


def _spins(sigma, n):
    s = np.ascontiguousarray(sigma, dtype=np.int8)
    if s.shape[-1] != n or not np.all(np.abs(s) == 1):
        raise ValueError("spins must be +-1 with the instance's length")
    return s


def energy(inst: Instance, sigma) -> float:
    """Exact E = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i, rounded once (Eq. 2, pairs once)."""
    s = _spins(sigma, inst.n)
    c = inst._c()
    return _load().or_energy(ctypes.byref(c), _ptr(s))


def energies(inst: Instance, sigmas) -> np.ndarray:
    s = np.atleast_2d(_spins(sigmas, inst.n))
    return np.array([energy(inst, row) for row in s])


def energy_quadratic(inst: Instance, sigma) -> float:
    """The same energy as (1/2) s^T J s + h.s in plain double arithmetic."""
    s = _spins(sigma, inst.n)
    c = inst._c()
    return _load().or_energy_quadratic(ctypes.byref(c), _ptr(s))


def cut(inst: Instance, sigma) -> float:
    """Exact cut weight: sum of w_ij over pairs i<j on opposite sides (Eq. 3)."""
    s = _spins(sigma, inst.n)
    c = inst._c()
    return _load().or_cut(ctypes.byref(c), _ptr(s))


def exact_sum(x) -> float:
    a = np.ascontiguousarray(x, dtype=np.float64)
    return _load().or_exact_sum(_ptr(a), a.size)


def local_field(inst: Instance, s, i: int) -> float:
    a = np.ascontiguousarray(s, dtype=np.float64)
    c = inst._c()
    return _load().or_local_field(ctypes.byref(c), _ptr(a), int(i))


def bruteforce(inst: Instance, tol: float = 0.0):
    """(E_min, one minimiser, number of minimisers) over all 2^n states (n <= 30)."""
    e = ctypes.c_double()
    cnt = ctypes.c_int64()
    s = np.zeros(inst.n, dtype=np.int8)
    c = inst._c()
    rc = _load().or_bruteforce(ctypes.byref(c), float(tol), ctypes.addressof(e), _ptr(s),
                               ctypes.addressof(cnt))
    if rc != 0:
        raise ValueError("bruteforce rejected the instance")
    return e.value, s, cnt.value


class Schedule(ctypes.Structure):
    """or_schedule: the paper's linear cooling when geometric and quench are 0."""
    _fields_ = [("geometric", ctypes.c_int32), ("ratio", ctypes.c_double),
                ("t_floor", ctypes.c_double), ("quench", ctypes.c_int32)]


def mars_solve(inst: Instance, m0, t0, *, c_step=1.0, d_min=1e-4, k_max=1000, fixed_sweeps=0,
               update=UPDATE_GS, order=None, nthreads=1, want_m=True, geometric=None,
               t_floor=0.0, quench=False):
    """Run Algorithm 1 for every replica; returns a dict of per-replica results.

    geometric=r (0 < r < 1) cools T <- r T while T > t_floor instead of the
    paper's T <- T - c_step; quench=True adds the final T -> 0+ level
    (s_i <- -sgn(Phi_i)). Both are labelled variants, off by default."""
    m0 = np.ascontiguousarray(m0, dtype=np.float32)
    t0 = np.ascontiguousarray(t0, dtype=np.float32)
    R = t0.shape[0]
    if m0.shape != (R, inst.n):
        raise ValueError("m0 must have shape (R, n)")
    order_a = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    if order_a is not None and sorted(order_a.tolist()) != list(range(inst.n)):
        raise ValueError("order must be a permutation of 0..n-1")
    m_out = np.zeros((R, inst.n), dtype=np.float64) if want_m else None
    sig = np.zeros((R, inst.n), dtype=np.int8)
    en = np.zeros(R, dtype=np.float64)
    st = (ReplicaStats * max(R, 1))()
    c = inst._c()
    sch = Schedule(1 if geometric else 0, float(geometric or 0.0), float(t_floor), 1 if quench else 0)
    rc = _load().or_mars_solve(ctypes.byref(c), _ptr(order_a), R, _ptr(m0), _ptr(t0),
                               float(c_step), float(d_min), int(k_max), int(fixed_sweeps),
                               int(update), ctypes.byref(sch), int(nthreads), _ptr(m_out), _ptr(sig),
                               _ptr(en), ctypes.addressof(st))
    if rc != 0:
        raise ValueError("oracle rejected the inputs")
    stats = {k: np.array([getattr(st[r], k) for r in range(R)])
             for k in ("sweeps", "levels", "capped_levels", "final_T", "last_d")}
    return {"m": m_out, "sigma": sig, "energy": en, **stats}


def nmfa_solve(inst: Instance, m0, t0, *, c_step=1.0, alpha=0.5, sigma=0.0, seed=0, stream=0,
               nthreads=1, want_m=True, geometric=None, t_floor=0.0):
    """Noisy mean-field annealing (Section 2) for every replica: synchronous
    normalised-field updates with Gaussian noise and alpha-mixing, one
    iteration per temperature level (see mars_oracle.h)."""
    m0 = np.ascontiguousarray(m0, dtype=np.float32)
    t0 = np.ascontiguousarray(t0, dtype=np.float32)
    R = t0.shape[0]
    if m0.shape != (R, inst.n):
        raise ValueError("m0 must have shape (R, n)")
    m_out = np.zeros((R, inst.n), dtype=np.float64) if want_m else None
    sig = np.zeros((R, inst.n), dtype=np.int8)
    en = np.zeros(R, dtype=np.float64)
    st = (ReplicaStats * max(R, 1))()
    c = inst._c()
    sch = Schedule(1 if geometric else 0, float(geometric or 0.0), float(t_floor), 0)
    rc = _load().or_nmfa_solve(ctypes.byref(c), R, _ptr(m0), _ptr(t0), float(c_step), float(alpha),
                               float(sigma), int(seed) & (2**64 - 1), int(stream), ctypes.byref(sch),
                               int(nthreads), _ptr(m_out), _ptr(sig), _ptr(en), ctypes.addressof(st))
    if rc != 0:
        raise ValueError("oracle rejected the inputs")
    stats = {k: np.array([getattr(st[r], k) for r in range(R)])
             for k in ("sweeps", "levels", "capped_levels", "final_T", "last_d")}
    return {"m": m_out, "sigma": sig, "energy": en, **stats}


def nmfa_normal(seed: int, stream: int, r: int, k: int, i: int) -> float:
    """NMFA's standard normal for (replica r, iteration k, spin i) (see mars_oracle.h)."""
    return _load().or_nmfa_normal(int(seed) & (2**64 - 1), int(stream), int(r), int(k), int(i))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw_replicas(seed: int, R: int, n: int, t_min: float, t_max: float, *, stream: int = 0,
                  r0: int = 0):
    """The library's counter-based start-state draw, restated (see mars_oracle.h)."""
    m0 = np.zeros((R, n), dtype=np.float32)
    t0 = np.zeros(R, dtype=np.float32)
    _load().or_draw_replicas(int(seed) & (2**64 - 1), int(stream), int(r0), int(R), int(n),
                             float(t_min), float(t_max), _ptr(m0), _ptr(t0))
    return m0, t0
