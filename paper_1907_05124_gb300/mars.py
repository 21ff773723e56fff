"""Python binding of the MARS C ABI (include/mars.h): argument marshalling only.

Every step of the method runs in the CUDA library ``_lib/libmars.so``; this
module converts numpy arrays or torch CUDA tensors to pointers, calls the
``mars_*`` entry points through ``ctypes`` and wraps the results. There is no
fallback: if the library is missing, or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmars.so")

MARS_OK, MARS_EINVAL, MARS_ENOMEM, MARS_EAGAIN, MARS_ETIMEOUT, MARS_EDEVICE, MARS_ENOTFOUND = \
    0, -1, -2, -3, -4, -5, -6
MARS_ECANCELED = -7
MARS_I8, MARS_F32, MARS_F64 = 1, 2, 3
MARS_DEVICE_PTR = 1
MARS_POLISH_FP32 = 2
NOALLOC_SCRATCH_BYTES = 16 << 20  # MARS_NOALLOC_SCRATCH_BYTES
UPDATE = {"gs": 0, "jacobi": 1}
PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2}

_ERRNAMES = {MARS_EINVAL: "EINVAL", MARS_ENOMEM: "ENOMEM", MARS_EAGAIN: "EAGAIN",
             MARS_ETIMEOUT: "ETIMEOUT", MARS_EDEVICE: "EDEVICE", MARS_ENOTFOUND: "ENOTFOUND",
             MARS_ECANCELED: "ECANCELED"}


class MarsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("replicas", ctypes.c_int32), ("t_min", ctypes.c_double),
                ("t_max", ctypes.c_double), ("c_step", ctypes.c_double),
                ("d_min", ctypes.c_double), ("k_max", ctypes.c_int32),
                ("fixed_sweeps", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_uint32), ("update", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("m0", ctypes.c_void_p),
                ("t0", ctypes.c_void_p), ("flags", ctypes.c_uint32),
                ("schedule", ctypes.c_int32), ("cool_ratio", ctypes.c_double),
                ("t_floor", ctypes.c_double), ("quench", ctypes.c_int32),
                ("method", ctypes.c_int32), ("nmfa_alpha", ctypes.c_double),
                ("nmfa_sigma", ctypes.c_double)]


METHOD = {"mars": 0, "nmfa": 1}


def _method(p, method="mars", alpha=0.5, sigma=0.0):
    """Set the method on Params p: MARS (Algorithm 1) or NMFA (noisy mean-field
    annealing with mixing weight alpha and noise deviation sigma)."""
    p.method = METHOD[method]
    p.nmfa_alpha = float(alpha)
    p.nmfa_sigma = float(sigma)


def _schedule(p, geometric=None, t_floor=0.0, quench=False):
    """Set the labelled schedule variants on Params p (defaults: the paper's)."""
    p.schedule = 1 if geometric else 0
    p.cool_ratio = float(geometric) if geometric else 0.5
    p.t_floor = float(t_floor)
    p.quench = 1 if quench else 0


class Outputs(ctypes.Structure):
    _fields_ = [("energies", ctypes.c_void_p), ("spins", ctypes.c_void_p),
                ("m_final", ctypes.c_void_p), ("t0", ctypes.c_void_p),
                ("sweeps", ctypes.c_void_p), ("levels", ctypes.c_void_p),
                ("capped", ctypes.c_void_p), ("flags", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("best_energy", ctypes.c_double), ("best_energy_i64", ctypes.c_int64),
                ("best_cut", ctypes.c_double), ("best_replica", ctypes.c_int32),
                ("hits", ctypes.c_int32), ("mean_energy", ctypes.c_double),
                ("sweeps", ctypes.c_int64), ("spin_updates", ctypes.c_int64),
                ("levels", ctypes.c_int64), ("capped_levels", ctypes.c_int64),
                ("gpu_seconds", ctypes.c_double), ("descent_seconds", ctypes.c_double),
                ("energy_err_bound", ctypes.c_double),
                ("status", ctypes.c_int32), ("integer", ctypes.c_int32),
                ("gemm_seconds", ctypes.c_double), ("gemm_launches", ctypes.c_int64),
                ("gemm_flops", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("level_seconds", ctypes.c_double), ("level_launches", ctypes.c_int64),
                ("level_updates", ctypes.c_int64)]


class InstanceInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("dense", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("levels", ctypes.c_int32), ("integer", ctypes.c_int32),
                ("total_weight", ctypes.c_double), ("device_bytes", ctypes.c_int64)]


# Every symbol include/mars.h declares, with its ctypes signature.
P = ctypes.c_void_p
class Shape(ctypes.Structure):
    """mars_shape: an instance's launch shape (-1 = library default)."""
    _fields_ = [("sell_rt", ctypes.c_int32), ("sell_threads", ctypes.c_int32),
                ("sell_smem_table", ctypes.c_int32), ("tc_rpw", ctypes.c_int32),
                ("tc_overlap", ctypes.c_int32), ("tc_pair", ctypes.c_int32)]


SIGNATURES = {
    "mars_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t, P]),
    "mars_destroy": (None, [P]),
    "mars_last_error": (ctypes.c_char_p, [P]),
    "mars_instance_dense": (ctypes.c_int, [P, ctypes.c_int32, P, ctypes.c_int32, P, P,
                                           ctypes.c_uint32, P]),
    "mars_instance_csr": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int64, P, P, P,
                                         ctypes.c_int32, P, P, ctypes.c_uint32, P]),
    "mars_instance_free": (ctypes.c_int, [P, ctypes.c_int32]),
    "mars_instance_get_info": (ctypes.c_int, [P, ctypes.c_int32, P]),
    "mars_instance_order": (ctypes.c_int, [P, ctypes.c_int32, P]),
    "mars_params_default": (None, [P]),
    "mars_solve": (ctypes.c_int, [P, ctypes.c_int32, P, P, P, P]),
    "mars_energy": (ctypes.c_int, [P, ctypes.c_int32, P, ctypes.c_int32, P, P,
                                   ctypes.c_uint32]),
    "mars_draw_replicas": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, P, P, ctypes.c_uint32]),
    "mars_solve_noalloc": (ctypes.c_int, [P, ctypes.c_int32, P, P, P, P]),
    "mars_solve_batch": (ctypes.c_int, [P, ctypes.c_int32, P, P, P, P]),
    "mars_serve_limits": (ctypes.c_int, [P, ctypes.c_int32]),
    "mars_submit": (ctypes.c_int, [P, ctypes.c_int32, P, P]),
    "mars_poll": (ctypes.c_int, [P, ctypes.c_int64, P, P]),
    "mars_serve_status": (ctypes.c_int, [P, P, P]),
    "mars_serve_counters": (ctypes.c_int, [P, P, P]),
    "mars_cancel": (ctypes.c_int, [P, ctypes.c_int64]),
    "mars_device_check": (ctypes.c_int, [P, ctypes.c_int32]),
    "mars_set_shape": (ctypes.c_int, [P, ctypes.c_int32, P]),
    "mars_get_shape": (ctypes.c_int, [P, ctypes.c_int32, P]),
    "mars_autotune": (ctypes.c_int, [P, ctypes.c_int32, P, ctypes.c_int32, P, P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"MARS CUDA library not built: {path} is missing "
                               "(run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _arr(x, dtype):
    """(pointer, keepalive, is_device) for a numpy array or torch tensor, or None."""
    if x is None:
        return None, None, False
    if _is_torch(x):
        import torch
        t = x.contiguous()
        want = {np.float32: torch.float32, np.float64: torch.float64, np.int8: torch.int8,
                np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if t.dtype != want:
            t = t.to(want)
        if not t.is_cuda:
            a = np.ascontiguousarray(t.numpy(), dtype=dtype)
            return a.ctypes.data, a, False
        return t.data_ptr(), t, True
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a, False


def _jtype(x):
    dt = str(getattr(x, "dtype", ""))
    if "int8" in dt:
        return MARS_I8, np.int8
    if "float32" in dt:
        return MARS_F32, np.float32
    return MARS_F64, np.float64


@dataclass
class SolveResult:
    best_energy: float
    best_energy_i64: int
    best_cut: float
    best_replica: int
    hits: int
    mean_energy: float
    sweeps: int
    spin_updates: int
    levels: int
    capped_levels: int
    gpu_seconds: float
    descent_seconds: float
    energy_err_bound: float
    integer: bool
    best_spins: np.ndarray
    gemm_seconds: float = 0.0
    gemm_launches: int = 0
    gemm_flops: float = 0.0
    kernel_launches: int = 0
    level_seconds: float = 0.0
    level_launches: int = 0
    level_updates: int = 0
    energies: np.ndarray | None = None
    spins: np.ndarray | None = None
    m_final: np.ndarray | None = None
    t0: np.ndarray | None = None
    replica_sweeps: np.ndarray | None = None
    replica_levels: np.ndarray | None = None
    replica_capped: np.ndarray | None = None


class Context:
    """A MARS context on one CUDA device (see mars_create)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, stream=None):
        self._lib = load()
        self.torch_stream = None
        if stream is None:
            # A dedicated torch stream (the legacy default stream has handle 0,
            # which the C ABI reads as "create your own"); callers order their
            # own work against ctx.torch_stream.
            try:
                import torch
                if torch.cuda.is_available():
                    self.torch_stream = torch.cuda.Stream(device)
                    stream = self.torch_stream.cuda_stream
            except ImportError:
                stream = None
        self._ctx = P()
        rc = self._lib.mars_create(ctypes.byref(self._ctx), int(device), int(hbm_budget_bytes),
                                   stream or None)
        if rc != MARS_OK:
            raise MarsError(rc, "mars_create failed (no usable CUDA device?)")
        self._n = {}

    def _after_current(self):
        """Order the library's stream after work already queued on torch's current stream."""
        if self.torch_stream is not None:
            import torch
            self.torch_stream.wait_stream(torch.cuda.current_stream())

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.mars_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != MARS_OK:
            raise MarsError(rc, self._lib.mars_last_error(self._ctx).decode())

    # -- instances ------------------------------------------------------------
    def add_dense(self, J, h=None, order=None) -> int:
        jt, dt = _jtype(J)
        n = int(J.shape[0])
        pj, kj, dev = _arr(J, dt)
        ph, kh, _ = _arr(None if h is None else np.asarray(h, np.float64), np.float64)
        po, ko, _ = _arr(None if order is None else np.asarray(order, np.int32), np.int32)
        if dev:
            self._after_current()
        inst = ctypes.c_int32()
        self._check(self._lib.mars_instance_dense(self._ctx, n, pj, jt, ph, po,
                                                  MARS_DEVICE_PTR if dev else 0,
                                                  ctypes.byref(inst)))
        self._n[inst.value] = n
        return inst.value

    def add_csr(self, row_ptr, col, val, h=None, order=None) -> int:
        vt, dt = _jtype(val)
        n = int(row_ptr.shape[0]) - 1
        nnz = int(col.shape[0])
        pr, kr, dev = _arr(row_ptr, np.int32)
        pc, kc, _ = _arr(col, np.int32)
        pv, kv, _ = _arr(val, dt)
        ph, kh, _ = _arr(None if h is None else np.asarray(h, np.float64), np.float64)
        po, ko, _ = _arr(None if order is None else np.asarray(order, np.int32), np.int32)
        if dev:
            self._after_current()
        inst = ctypes.c_int32()
        self._check(self._lib.mars_instance_csr(self._ctx, n, nnz, pr, pc, pv, vt, ph, po,
                                                MARS_DEVICE_PTR if dev else 0,
                                                ctypes.byref(inst)))
        self._n[inst.value] = n
        return inst.value

    def free(self, inst: int):
        self._check(self._lib.mars_instance_free(self._ctx, int(inst)))
        self._n.pop(inst, None)

    def info(self, inst: int) -> dict:
        i = InstanceInfo()
        self._check(self._lib.mars_instance_get_info(self._ctx, int(inst), ctypes.byref(i)))
        return {k: getattr(i, k) for k, _ in InstanceInfo._fields_}

    def order(self, inst: int) -> np.ndarray:
        o = np.zeros(self._n[inst], dtype=np.int32)
        self._check(self._lib.mars_instance_order(self._ctx, int(inst), o.ctypes.data))
        return o

    # -- solve ----------------------------------------------------------------
    def solve(self, inst: int, replicas: int, t_min: float, t_max: float, *, c_step=1.0,
              d_min=1e-4, k_max=1000, fixed_sweeps=0, seed=0, stream=0, update="gs",
              precision="fp32", m0=None, t0=None, outputs=("energies",), device_outputs=False,
              polish=False, geometric=None, t_floor=0.0, quench=False, method="mars", alpha=0.5,
              sigma=0.0):
        """Run mars_solve; `outputs` names the per-replica arrays to return.
        geometric=r (with t_floor) and quench=True select the labelled
        schedule variants (the paper's linear schedule by default);
        method="nmfa" runs noisy mean-field annealing with alpha and sigma."""
        n = self._n[inst]
        p = Params()
        self._lib.mars_params_default(ctypes.byref(p))
        _schedule(p, geometric, t_floor, quench)
        _method(p, method, alpha, sigma)
        p.replicas, p.t_min, p.t_max, p.c_step, p.d_min = int(replicas), t_min, t_max, c_step, d_min
        p.k_max, p.fixed_sweeps, p.seed, p.stream = int(k_max), int(fixed_sweeps), int(seed), int(stream)
        p.update, p.precision = UPDATE[update], PRECISION[precision]
        pm, km, dm = _arr(m0, np.float32)
        pt, kt, dt_ = _arr(t0, np.float32)
        if m0 is not None and t0 is not None and dm != dt_:
            raise ValueError("m0 and t0 must both be host arrays or both device tensors")
        p.m0, p.t0 = pm, pt
        p.flags = (MARS_DEVICE_PTR if (dm or dt_) else 0) | (MARS_POLISH_FP32 if polish else 0)
        R = int(replicas)
        want = set(outputs or ())
        o = Outputs()
        keep = {}
        if device_outputs:
            import torch
            shapes = {"energies": ((R,), torch.float64), "spins": ((R, n), torch.int8),
                      "m_final": ((R, n), torch.float32), "t0": ((R,), torch.float32),
                      "sweeps": ((R,), torch.int32), "levels": ((R,), torch.int32),
                      "capped": ((R,), torch.int32)}
            for k in want:
                keep[k] = torch.empty(shapes[k][0], dtype=shapes[k][1], device="cuda")
                setattr(o, k, keep[k].data_ptr())
            o.flags = MARS_DEVICE_PTR
        else:
            shapes = {"energies": ((R,), np.float64), "spins": ((R, n), np.int8),
                      "m_final": ((R, n), np.float32), "t0": ((R,), np.float32),
                      "sweeps": ((R,), np.int32), "levels": ((R,), np.int32),
                      "capped": ((R,), np.int32)}
            for k in want:
                keep[k] = np.zeros(shapes[k][0], dtype=shapes[k][1])
                setattr(o, k, keep[k].ctypes.data)
        if dm or dt_ or device_outputs:
            self._after_current()
        best = np.zeros(n, dtype=np.int8)
        res = Result()
        self._check(self._lib.mars_solve(self._ctx, int(inst), ctypes.byref(p), best.ctypes.data,
                                         ctypes.byref(o), ctypes.byref(res)))
        return SolveResult(
            best_energy=res.best_energy, best_energy_i64=res.best_energy_i64,
            best_cut=res.best_cut, best_replica=res.best_replica, hits=res.hits,
            mean_energy=res.mean_energy, sweeps=res.sweeps, spin_updates=res.spin_updates,
            levels=res.levels, capped_levels=res.capped_levels, gpu_seconds=res.gpu_seconds,
            descent_seconds=res.descent_seconds,
            energy_err_bound=res.energy_err_bound, integer=bool(res.integer), best_spins=best,
            gemm_seconds=res.gemm_seconds, gemm_launches=res.gemm_launches,
            gemm_flops=res.gemm_flops, kernel_launches=res.kernel_launches,
            level_seconds=res.level_seconds, level_launches=res.level_launches,
            level_updates=res.level_updates, energies=keep.get("energies"), spins=keep.get("spins"), m_final=keep.get("m_final"),
            t0=keep.get("t0"), replica_sweeps=keep.get("sweeps"),
            replica_levels=keep.get("levels"), replica_capped=keep.get("capped"))

    # -- launch shape and autotuner -------------------------------------------
    def set_shape(self, inst: int, **shape):
        """mars_set_shape: sell_rt, sell_threads, sell_smem_table, tc_rpw,
        tc_overlap, tc_pair (omitted = -1, the default); no keywords clears the shape."""
        unknown = set(shape) - {k for k, _ in Shape._fields_}
        if unknown:
            raise ValueError(f"unknown launch-shape keys {sorted(unknown)}")
        if not shape:
            self._check(self._lib.mars_set_shape(self._ctx, int(inst), None))
            return
        sh = Shape(*[int(shape.get(k, -1)) for k, _ in Shape._fields_])
        self._check(self._lib.mars_set_shape(self._ctx, int(inst), ctypes.byref(sh)))

    def get_shape(self, inst: int) -> dict:
        sh = Shape()
        self._check(self._lib.mars_get_shape(self._ctx, int(inst), ctypes.byref(sh)))
        return {k: getattr(sh, k) for k, _ in Shape._fields_}

    def autotune(self, inst: int, replicas: int, t_min: float, t_max: float, *, repeats=3,
                 c_step=1.0, d_min=1e-4, k_max=1000, fixed_sweeps=0, seed=0, stream=0,
                 update="gs", precision="fp32", m0=None, t0=None):
        """mars_autotune with these solve parameters (host m0/t0 only).
        Returns (shape dict stored on the instance, fastest descent seconds)."""
        p = Params()
        self._lib.mars_params_default(ctypes.byref(p))
        p.replicas, p.t_min, p.t_max, p.c_step, p.d_min = int(replicas), t_min, t_max, c_step, d_min
        p.k_max, p.fixed_sweeps, p.seed, p.stream = int(k_max), int(fixed_sweeps), int(seed), int(stream)
        p.update, p.precision = UPDATE[update], PRECISION[precision]
        pm, km, dm = _arr(None if m0 is None else np.asarray(m0, np.float32), np.float32)
        pt, kt, dt_ = _arr(None if t0 is None else np.asarray(t0, np.float32), np.float32)
        p.m0, p.t0 = pm, pt
        sh = Shape()
        sec = ctypes.c_double()
        self._check(self._lib.mars_autotune(self._ctx, int(inst), ctypes.byref(p), int(repeats),
                                            ctypes.byref(sh), ctypes.byref(sec)))
        return {k: getattr(sh, k) for k, _ in Shape._fields_}, sec.value

    def solve_batch(self, jobs):
        """mars_solve_batch over [(inst, replicas, t_min, t_max, kwargs), ...].

        kwargs may hold c_step, d_min, k_max, fixed_sweeps, seed, stream, m0, t0
        (host arrays). Returns a list of SolveResult (best spins and summary).
        """
        cnt = len(jobs)
        params = (Params * cnt)()
        insts = (ctypes.c_int32 * cnt)()
        keep = []
        bests = []
        for j, (inst, R, t_min, t_max, kw) in enumerate(jobs):
            p = params[j]
            self._lib.mars_params_default(ctypes.byref(p))
            p.replicas, p.t_min, p.t_max = int(R), float(t_min), float(t_max)
            p.c_step = float(kw.get("c_step", 1.0))
            p.d_min = float(kw.get("d_min", 1e-4))
            p.k_max = int(kw.get("k_max", 1000))
            p.fixed_sweeps = int(kw.get("fixed_sweeps", 0))
            p.seed = int(kw.get("seed", 0))
            p.stream = int(kw.get("stream", 0))
            _schedule(p, kw.get("geometric"), kw.get("t_floor", 0.0), kw.get("quench", False))
            pm, km, _ = _arr(kw.get("m0"), np.float32)
            pt, kt, _ = _arr(kw.get("t0"), np.float32)
            p.m0, p.t0 = pm, pt
            keep += [km, kt]
            insts[j] = int(inst)
            bests.append(np.zeros(self._n[inst], dtype=np.int8))
        ptrs = (ctypes.c_void_p * cnt)(*[b.ctypes.data for b in bests])
        res = (Result * cnt)()
        self._check(self._lib.mars_solve_batch(self._ctx, cnt, insts, params, ptrs, res))
        out = []
        for j in range(cnt):
            r = res[j]
            out.append(SolveResult(
                best_energy=r.best_energy, best_energy_i64=r.best_energy_i64,
                best_cut=r.best_cut, best_replica=r.best_replica, hits=r.hits,
                mean_energy=r.mean_energy, sweeps=r.sweeps, spin_updates=r.spin_updates,
                levels=r.levels, capped_levels=r.capped_levels, gpu_seconds=r.gpu_seconds,
                descent_seconds=r.descent_seconds, energy_err_bound=r.energy_err_bound,
                integer=bool(r.integer), best_spins=bests[j], kernel_launches=r.kernel_launches))
        return out

    # -- serving ------------------------------------------------------------------
    def serve_limits(self, max_inflight: int):
        self._check(self._lib.mars_serve_limits(self._ctx, int(max_inflight)))

    def submit(self, inst: int, replicas: int, t_min: float, t_max: float, *, c_step=1.0,
               d_min=1e-4, k_max=1000, fixed_sweeps=0, seed=0, stream=0, update="gs",
               precision="fp32", geometric=None, t_floor=0.0, quench=False, method="mars",
               alpha=0.5, sigma=0.0) -> int:
        """mars_submit: queue a solve and return its request id."""
        p = Params()
        self._lib.mars_params_default(ctypes.byref(p))
        _schedule(p, geometric, t_floor, quench)
        _method(p, method, alpha, sigma)
        p.replicas, p.t_min, p.t_max, p.c_step, p.d_min = int(replicas), t_min, t_max, c_step, d_min
        p.k_max, p.fixed_sweeps, p.seed, p.stream = int(k_max), int(fixed_sweeps), int(seed), int(stream)
        p.update, p.precision = UPDATE[update], PRECISION[precision]
        req = ctypes.c_int64()
        self._check(self._lib.mars_submit(self._ctx, int(inst), ctypes.byref(p), ctypes.byref(req)))
        self._req_n = getattr(self, "_req_n", {})
        self._req_n[req.value] = self._n[inst]
        return req.value

    def poll(self, req: int):
        """mars_poll: None while pending, else a SolveResult (raises if the request failed)."""
        n = self._req_n[req]
        best = np.zeros(n, dtype=np.int8)
        r = Result()
        rc = self._lib.mars_poll(self._ctx, int(req), best.ctypes.data, ctypes.byref(r))
        if rc == MARS_EAGAIN:
            return None
        self._req_n.pop(req, None)
        self._check(rc)
        return SolveResult(
            best_energy=r.best_energy, best_energy_i64=r.best_energy_i64, best_cut=r.best_cut,
            best_replica=r.best_replica, hits=r.hits, mean_energy=r.mean_energy, sweeps=r.sweeps,
            spin_updates=r.spin_updates, levels=r.levels, capped_levels=r.capped_levels,
            gpu_seconds=r.gpu_seconds, descent_seconds=r.descent_seconds,
            energy_err_bound=r.energy_err_bound, integer=bool(r.integer), best_spins=best)

    def serve_counters(self):
        """(requests served by the persistent serving kernel, requests on their own streams)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.mars_serve_counters(self._ctx, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def cancel(self, req: int):
        """mars_cancel: drop a queued request, or discard a running one's results."""
        self._check(self._lib.mars_cancel(self._ctx, int(req)))

    def device_check(self, budget_us: int = 100000):
        """mars_device_check: a bounded device wait on a host-mapped flag (raises
        MarsError with MARS_ETIMEOUT when the wait gives up)."""
        self._check(self._lib.mars_device_check(self._ctx, int(budget_us)))

    def serve_status(self):
        q, rn = ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.mars_serve_status(self._ctx, ctypes.byref(q), ctypes.byref(rn)))
        return q.value, rn.value

    def energy(self, inst: int, spins):
        """Exact energies of spin vectors (count, n) or (n,) -> (float64[count], int64[count])."""
        n = self._n[inst]
        s = np.atleast_2d(np.ascontiguousarray(spins, dtype=np.int8))
        if s.shape[1] != n:
            raise ValueError("spins must have the instance's length")
        cnt = s.shape[0]
        e = np.zeros(cnt, dtype=np.float64)
        ei = np.zeros(cnt, dtype=np.int64)
        self._check(self._lib.mars_energy(self._ctx, int(inst), s.ctypes.data, cnt, e.ctypes.data,
                                          ei.ctypes.data, 0))
        return e, ei

    def draw_replicas(self, seed: int, R: int, n: int, t_min: float, t_max: float, *, stream=0,
                      r0=0):
        m0 = np.zeros((R, n), dtype=np.float32)
        t0 = np.zeros(R, dtype=np.float32)
        self._check(self._lib.mars_draw_replicas(self._ctx, int(seed), int(stream), int(r0), int(R),
                                                 int(n), float(t_min), float(t_max), m0.ctypes.data,
                                                 t0.ctypes.data, 0))
        return m0, t0
