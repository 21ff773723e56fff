#!/usr/bin/env python
"""MARS benchmark: spin-updates/s on dense SK N=8192 with BF16 tensor cores.

Workload (one step, the default): a dense Sherrington-Kirkpatrick instance with
N = 8192 spins and J_ij ~ Normal(0, 1/N) (symmetric, zero diagonal, h = 0,
seed 0), R = 4096 replicas with start states and start temperatures
T0 ~ U(0, 2) drawn on the device, linear cooling C_step = 1/sqrt(N),
d_min = 1e-4, k_max = 1000, sequential sweeps whose panel fields come from
BF16 tcgen05 GEMMs with FP32 accumulation; then sign-rounding, exact FP64
energies and the best replica. One step is one whole mars_solve.

A spin-update is one new s_i of one replica in one sweep; the metric counts
only the sweeps replicas actually perform. The line also carries the time to
target energy against the plain FP32 path (vs_fp32_path), measured in the same
run on a smaller instance of the same family that both paths finish quickly.

Other workloads (--workload): ea2d (2-D +-J lattice L=100, R=1024), ea3d_big
(3-D lattice N=10^6, magnetisations in HBM), sk8192pm1 (the FP8 variant),
batch, serve, ttt, sensitivity.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mars|reference]

With --gpus N > 1 launch under torch.distributed.run; every rank solves its
own R replicas (a different Philox stream), there is no data-path collective
(weak scaling). --impl reference times the FP64 CPU oracle on the host cores
for the same workload and metric (a bounded sample of replicas per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L, R, T_MIN, T_MAX = 100, 1024, 0.0, 4.0
C_STEP, D_MIN, K_MAX = 1.0, 1e-4, 1000
WORKLOAD = {
    "workload": "2-D EA +-J spin glass, periodic 100x100 (N=10000), R=1024 replicas, "
                "T0~U(0,4), C_step=1, d_min=1e-4, k_max=1000, FP32 sequential sweeps "
                "in colour order",
    "n_spins": L * L, "replicas": R, "t_range": [T_MIN, T_MAX], "c_step": C_STEP,
    "d_min": D_MIN, "k_max": K_MAX,
}
# Dense SK with Gaussian couplings on the tensor cores (BF16 J*m, FP32 fields).
SK_N, SK_R, SK_TMAX = 8192, 4096, 2.0
SK_WORKLOAD = {
    "workload": "dense SK N=8192, J_ij ~ Normal(0, 1/N), R=4096 replicas, T0~U(0,2), "
                "C_step=1/sqrt(N), d_min=1e-4, k_max=1000, sequential sweeps with BF16 "
                "tcgen05 panel GEMMs",
    "n_spins": SK_N, "replicas": SK_R, "t_range": [0.0, SK_TMAX], "c_step": 1.0 / SK_N ** 0.5,
    "d_min": D_MIN, "k_max": K_MAX, "precision": "bf16",
}

# A sparse instance too large for shared memory: the 3-D lattice L=100, whose
# replicas' magnetisations all stay resident in HBM while each level of a
# sweep is spread over the whole GPU.
EA3_L, EA3_R, EA3_TMAX = 100, 608, 6.0
EA3_WORKLOAD = {
    "workload": "3-D EA +-J spin glass, periodic 100^3 (N=1,000,000), R=608 replicas, "
                "T0~U(0,6), C_step=1, d_min=1e-4, k_max=1000, FP32 sequential sweeps in colour "
                "order, every replica's magnetisations resident in HBM, one grid-wide launch per "
                "colour level",
    "n_spins": EA3_L ** 3, "replicas": EA3_R, "t_range": [0.0, EA3_TMAX], "c_step": 1.0,
    "d_min": D_MIN, "k_max": K_MAX,
}
# Algorithmic DRAM bytes per spin-update of a two-colour sweep whose slabs are
# far larger than L2: every magnetisation is read twice per sweep (as the
# other colour's neighbour and as its own old value) and written once.
EA3_BYTES_PER_UPDATE = 12.0
# DRAM bytes per live spin-update of the staged level kernel, from one ncu
# capture of a launch of the N=10^6 lattice (dram__bytes_read.sum +
# dram__bytes_write.sum = 3.328 GB for 510 live replicas x 500,000 spins).
EA3_DRAM_BYTES_PER_UPDATE = 3.328e9 / (510 * 500_000)

# The FP8 variant: dense SK with +-1 couplings (exact in E4M3) on E4M3 tensor
# cores; the same schedule in units of the couplings' scale sqrt(N).
SK8_TMAX = 2.0 * SK_N ** 0.5
SK8_WORKLOAD = {
    "workload": "dense SK N=8192, J_ij uniform in {-1,+1}, R=4096 replicas, T0~U(0,2 sqrt(N)), "
                "C_step=1, d_min=1e-4, k_max=1000, sequential sweeps with FP8 (E4M3) "
                "tcgen05 panel GEMMs",
    "n_spins": SK_N, "replicas": SK_R, "t_range": [0.0, SK8_TMAX], "c_step": 1.0,
    "d_min": D_MIN, "k_max": K_MAX, "precision": "fp8",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mars", choices=["mars", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip mars_autotune before the warm-up (library default launch shape)")
    ap.add_argument("--workload", default="sk8192",
                    choices=["ea2d", "ea3d_big", "sk8192", "sk8192pm1", "serve", "ttt", "batch",
                             "sensitivity"],
                    help="sk8192: dense SK N=8192 on BF16 tensor cores (default); ea2d: the 2-D "
                         "lattice L=100; ea3d_big: the 3-D lattice with N=10^6 (magnetisations in "
                         "HBM); sk8192pm1: the +-1 variant on FP8 tensor cores; "
                         "serve: Poisson arrivals of mixed requests through mars_submit/mars_poll")
    ap.add_argument("--requests", type=int, default=2000, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=1.5,
                    help="serve: mean arrivals per second")
    ap.add_argument("--inflight", type=int, default=16,
                    help="serve: requests admitted at once (mars_serve_limits)")
    ap.add_argument("--serve-deadline", type=float, default=1500.0,
                    help="serve: seconds after which requests still pending are cancelled "
                         "(counted in the line, excluded from the latencies)")
    ap.add_argument("--replicas", type=int, default=0, help="override R (profiling runs)")
    ap.add_argument("--fixed-sweeps", type=int, default=0,
                    help="profiling runs only: exactly this many sweeps per level")
    ap.add_argument("--no-fp32-comparison", action="store_true",
                    help="skip the time-to-target comparison with the FP32 path")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_dense_sample(O, inst, wl, count, r0):
    """The oracle on `count` replicas of a dense workload (start states from the
    library's draw, replicas r0..r0+count-1), each doing 4 sweeps at one level
    (its start temperature moved into (C_step, 2 C_step]): the cost of a dense
    sweep does not depend on T. Returns (seconds, spin-updates)."""
    import numpy as np
    m0, t0 = O.draw_replicas(0, count, wl.J.shape[0], T_MIN, wl.t_max, r0=r0)
    t0 = (wl.c_step * (1.0 + np.clip(t0 / wl.t_max, 0.01, 1.0))).astype(np.float32)
    t = time.perf_counter()
    out = O.mars_solve(inst, m0, t0, c_step=wl.c_step, d_min=D_MIN, k_max=K_MAX, fixed_sweeps=4,
                       nthreads=count, want_m=False)
    return time.perf_counter() - t, int(out["sweeps"].sum()) * wl.J.shape[0]


def cpu_baseline(target_s: float, wl=None):
    """The FP64 oracle on the host cores, on a bounded sample of the same workload."""
    import numpy as np

    import oracle as O
    from paper_1907_05124_gb300 import instances as I

    cores = os.cpu_count() or 1
    if wl is not None and wl.name in ("sk8192", "sk8192pm1"):
        # A dense N=8192 sweep costs ~0.4 s on one core, whatever its
        # temperature: time batches of one replica per core, 4 sweeps each,
        # until the target CPU time is spent.
        inst = O.Instance.dense(wl.J)
        t_used, upd, k = 0.0, 0, 0
        while t_used < target_s:
            dt, u = oracle_dense_sample(O, inst, wl, cores, k * cores)
            t_used, upd, k = t_used + dt, upd + u, k + 1
        return {"value": upd / t_used, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{k * cores} replicas of the N=8192 workload, 4 sweeps each at one level, "
                          f"FP64 oracle, OpenMP over replicas, {t_used:.1f} s"}
    if wl is not None and wl.name == "ea3d_big":
        # One replica per core of the N=10^6 lattice, one sweep per level.
        inst = O.Instance.csr(wl.csr)
        order = I.greedy_colour_order(wl.csr)
        m0, t0 = O.draw_replicas(0, cores, wl.csr.n, T_MIN, wl.t_max)
        t = time.perf_counter()
        out = O.mars_solve(inst, m0, t0, c_step=wl.c_step, d_min=D_MIN, k_max=K_MAX, order=order,
                           fixed_sweeps=1, nthreads=cores, want_m=False)
        dt = time.perf_counter() - t
        upd = int(out["sweeps"].sum()) * wl.csr.n
        return {"value": upd / dt, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{cores} replicas of the N=10^6 lattice workload, one sweep per level, "
                          f"FP64 oracle, OpenMP over replicas, {dt:.1f} s"}
    csr = I.ea_lattice(L, 2, 0)
    inst = O.Instance.csr(csr)
    order = I.greedy_colour_order(csr)
    done_r, upd, t_used = 0, 0, 0.0
    batch = cores
    while t_used < target_s and done_r < R:
        b = min(batch, R - done_r)
        m0, t0 = O.draw_replicas(0, b, csr.n, T_MIN, T_MAX, r0=done_r)
        t = time.perf_counter()
        out = O.mars_solve(inst, m0, t0, c_step=C_STEP, d_min=D_MIN, k_max=K_MAX, order=order,
                           nthreads=cores, want_m=False)
        t_used += time.perf_counter() - t
        upd += int(out["sweeps"].sum()) * csr.n
        done_r += b
    return {"value": upd / t_used, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"replicas 0..{done_r - 1} of the R=1024 workload (seed 0), FP64 oracle, "
                      f"OpenMP over replicas, {t_used:.1f} s"}


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle, each step a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle as O
    from paper_1907_05124_gb300 import instances as I
    O.build()
    cores = os.cpu_count() or 1
    per_step = cores  # replicas per step: one per host thread
    wl = Workload(args, 0)
    if wl.J is not None:
        inst = O.Instance.dense(wl.J)
        what = f"{per_step} replicas per step, 4 sweeps each at one level"

        def step(k):
            return oracle_dense_sample(O, inst, wl, per_step, (k * per_step) % wl.R)
    else:
        csr = wl.csr
        inst = O.Instance.csr(csr)
        order = I.greedy_colour_order(csr)
        one_sweep = wl.name != "ea2d"  # the N=10^6 lattice: one sweep per level
        what = f"{per_step} replicas per step" + (", one sweep per level" if one_sweep else "")

        def step(k):
            m0, t0 = O.draw_replicas(0, per_step, csr.n, T_MIN, wl.t_max, r0=(k * per_step) % wl.R)
            t = time.perf_counter()
            out = O.mars_solve(inst, m0, t0, c_step=wl.c_step, d_min=D_MIN, k_max=K_MAX, order=order,
                               fixed_sweeps=1 if one_sweep else 0, nthreads=cores, want_m=False)
            return time.perf_counter() - t, int(out["sweeps"].sum()) * csr.n

    for w in range(args.warmup):
        step(1000 + w)
    tot_t, tot_u = 0.0, 0
    for k in range(args.steps):
        dt, u = step(k)
        tot_t += dt
        tot_u += u
    value = tot_u / tot_t
    line = {
        "impl": "reference", "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded instance, Philox start states)",
        "config": dict(wl.config, sample=what),
        "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{what} x {args.steps} steps"},
        "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def aggregate(tot_ms, updates, device):
    """Whole-job numbers across ranks: the slowest rank's time, all ranks' updates.

    Ranks solve disjoint replica sets (Philox stream = rank) of the same
    instance; nothing else is exchanged.
    """
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(tot_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d["bf16_tflops_sustained"], "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "source": "fallback"}


class Workload:
    """One benchmark workload: how to build the instance and call mars_solve."""

    def __init__(self, args, rank):
        from paper_1907_05124_gb300 import instances
        self.name = args.workload
        if self.name == "ea2d":
            self.csr = instances.ea_lattice(L, 2, 0)
            self.J = None
            self.R = args.replicas or R
            self.t_max, self.c_step, self.precision = T_MAX, C_STEP, "fp32"
            self.config = dict(WORKLOAD, replicas=self.R)
            self.dtype = "f32"
        elif self.name == "ea3d_big":
            self.csr = instances.ea_lattice(EA3_L, 3, 0)
            self.J = None
            self.R = args.replicas or EA3_R
            self.t_max, self.c_step, self.precision = EA3_TMAX, 1.0, "fp32"
            self.config = dict(EA3_WORKLOAD, replicas=self.R)
            self.dtype = "f32"
        elif self.name == "sk8192":
            self.csr = None
            self.J = instances.sk_gauss(SK_N, 0)
            self.R = args.replicas or SK_R
            self.t_max, self.c_step, self.precision = SK_TMAX, 1.0 / SK_N ** 0.5, "bf16"
            self.config = dict(SK_WORKLOAD, replicas=self.R)
            self.dtype = "bf16"
        else:
            self.csr = None
            self.J = instances.sk_pm1(SK_N, 0)
            self.R = args.replicas or SK_R
            self.t_max, self.c_step, self.precision = SK8_TMAX, 1.0, "fp8"
            self.config = dict(SK8_WORKLOAD, replicas=self.R)
            self.dtype = "e4m3"
        self.rank = rank
        self.fixed = args.fixed_sweeps
        if self.fixed:
            self.config = dict(self.config, fixed_sweeps=self.fixed, note="profiling run")

    def add(self, ctx):
        return ctx.add_csr(*self.csr) if self.csr is not None else ctx.add_dense(self.J)

    def autotune(self, ctx, inst):
        """mars_autotune on this workload's replicas: the full solve for the
        lattice (milliseconds), a two-level fixed-sweep schedule for the dense
        instance (its full solve takes minutes). Untimed, before the warm-up."""
        if self.name == "ea2d":
            return ctx.autotune(inst, self.R, T_MIN, self.t_max, repeats=2, c_step=self.c_step,
                                d_min=D_MIN, k_max=K_MAX, seed=7, stream=self.rank)
        if self.csr is not None:  # seconds per solve: two levels of two sweeps each
            return ctx.autotune(inst, self.R, 0.0, 2.0 * self.c_step, repeats=1, c_step=self.c_step,
                                fixed_sweeps=2, seed=7, stream=self.rank)
        return ctx.autotune(inst, self.R, 0.0, 2.0 * self.c_step, repeats=1, c_step=self.c_step,
                            fixed_sweeps=4, seed=7, stream=self.rank, precision=self.precision)

    def solve(self, ctx, inst, seed):
        return ctx.solve(inst, self.R, T_MIN, self.t_max, c_step=self.c_step, d_min=D_MIN,
                         k_max=K_MAX, seed=seed, stream=self.rank, precision=self.precision,
                         fixed_sweeps=self.fixed, outputs=())


def fp32_path_comparison(ctx, n=1024, R=256, seeds=range(10)):
    """Time to target energy of the BF16 tensor-core path against the plain
    FP32 SIMT path, on an instance of the default workload's family small
    enough for the FP32 path to finish in seconds: dense SK with
    J_ij ~ Normal(0, 1/N) (instances.sk_gauss(1024, 3)), T0 ~ U(0, 2),
    C_step = 1/sqrt(N), d_min = 1e-4, k_max = 1000.

    The target is the FP64 oracle's best energy on the instance with a large
    budget (1024 replicas), stored by tests/golden/make_sk_gauss1024_target.py.
    Each path runs one solve of R replicas for every seed 0-9; a seed's time
    to target is its solve's wall time when the solve's best energy is at or
    below the target (within 1e-9 relative), else it is not reached. The
    median over the seeds is reported when more than half reach the target;
    with P the fraction of all replicas that reach it and t the mean solve
    time, t ln(0.01) / ln(1 - P) (the time to reach it with probability 0.99)
    is reported beside it, and the speedup uses the median where both paths
    have one."""
    import numpy as np
    import torch

    from paper_1907_05124_gb300 import instances
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                           "sk_gauss1024_target.json")) as f:
        golden = json.load(f)
    target = float(golden["best_energy"])
    tol = 1e-9 * abs(target)
    inst = ctx.add_dense(instances.sk_gauss(n, 3))
    c = 1.0 / n ** 0.5
    out = {"workload": f"dense SK N={n}, J_ij ~ Normal(0, 1/N), R={R} per solve, T0~U(0,2), "
                       "C_step=1/sqrt(N), d_min=1e-4, k_max=1000, seeds 0-9 on both paths",
           "target": f"FP64 oracle's best over {golden['replicas']} replicas "
                     "(tests/golden/sk_gauss1024_target.json)",
           "target_energy": target}
    for prec in ("fp32", "bf16"):
        kw = dict(c_step=c, d_min=D_MIN, k_max=K_MAX, precision=prec, outputs=("energies",))
        ctx.solve(inst, R, 0.0, 2.0, seed=100, fixed_sweeps=1, **kw)  # warm-up (short)
        secs, hit, reached, upd = [], [], 0, 0
        for sd in seeds:
            torch.cuda.synchronize()
            t = time.perf_counter()
            res = ctx.solve(inst, R, 0.0, 2.0, seed=sd, **kw)
            secs.append(time.perf_counter() - t)
            hit.append(res.best_energy <= target + tol)
            reached += int(np.sum(res.energies <= target + tol))
            upd += res.spin_updates
        out[prec] = dict(ttt_summary(secs, hit, reached, R),
                         spin_updates_per_s=upd / float(np.sum(secs)))
    ctx.free(inst)
    out.update(ttt_speedup(out["fp32"], out["bf16"]))
    return out


def ttt_summary(secs, hit, reached, R):
    """Time to target of one path from its per-seed solves: secs[i] is seed
    i's solve time, hit[i] whether that solve's best reached the target, and
    reached the number of replicas (R per solve) that reached it. The median
    over seeds (a seed that missed counts as infinitely slow) when more than
    half the seeds hit (so that the median is finite), else None; and t ln(0.01) / ln(1 - P), the time to
    reach the target with probability 0.99 when a fraction P of replicas
    reach it in a solve of mean time t."""
    import numpy as np
    P = reached / (R * len(secs))
    t_sim = float(np.mean(secs))
    ttt99 = t_sim * np.log(0.01) / np.log1p(-P) if 0 < P < 1 else (t_sim if P >= 1 else float("inf"))
    ttt = sorted(s_ if h else float("inf") for s_, h in zip(secs, hit))
    med = float(np.median(ttt)) if sum(hit) * 2 > len(hit) else None
    return {"solve_s_mean": t_sim, "seeds_reaching_target": int(sum(hit)), "P": P,
            "ttt_median_s": med, "ttt99_s": float(ttt99)}


def ttt_speedup(slow, fast):
    """The speedup at equal time to target: from the medians when both paths
    have one, else from the probability form."""
    if slow["ttt_median_s"] is not None and fast["ttt_median_s"] is not None:
        return {"speedup_at_equal_ttt": slow["ttt_median_s"] / fast["ttt_median_s"],
                "speedup_from": "median over seeds 0-9"}
    sp = slow["ttt99_s"] / fast["ttt99_s"] if fast["ttt99_s"] > 0 else None
    return {"speedup_at_equal_ttt": sp, "speedup_from": "t ln(0.01) / ln(1 - P)"}


def run_mars(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1907_05124_gb300 import build, mars
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    wl = Workload(args, rank)
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(args.cpu_seconds, wl)  # before any GPU work: plain host threads

    ctx = mars.Context(local)
    inst = wl.add(ctx)
    info = ctx.info(inst)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    stream = ctx.torch_stream  # the stream every library call is ordered on

    shape = None
    if wl.J is not None:
        # dense tensor-core solves: the library re-plans every batch of sweeps
        # for the replicas still active, which a fixed shape tuned on a short
        # all-active run would switch off
        wl.config = dict(wl.config, launch_shape_by="library plan per batch of sweeps (active replicas)")
    elif not args.no_autotune:
        shape, _ = wl.autotune(ctx, inst)
        wl.config = dict(wl.config, launch_shape=shape, launch_shape_by="mars_autotune")
    for w in range(max(args.warmup, 0)):
        wl.solve(ctx, inst, 10_000 + w)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    step_ms, descent_s, updates, best = [], [], 0, []
    gemm_s, gemm_flops, gemm_launches, launches = 0.0, 0.0, 0, 0
    level_s, level_upd, level_launches = 0.0, 0, 0
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between timed steps, outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = wl.solve(ctx, inst, k)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        descent_s.append(res.descent_seconds)
        updates += res.spin_updates
        best.append(res.best_energy)
        gemm_s += res.gemm_seconds
        gemm_flops += res.gemm_flops
        gemm_launches += res.gemm_launches
        launches += res.kernel_launches
        level_s += res.level_seconds
        level_upd += res.level_updates
        level_launches += res.level_launches
    clocks = sampler.stop()
    torch.cuda.synchronize()
    tot_ms = sum(step_ms)
    if world > 1:
        tot_ms, updates_all = aggregate(tot_ms, updates, "cuda")
        torch.distributed.barrier()
    else:
        updates_all = updates
    value = updates_all / (tot_ms * 1e-3)

    # End to end through the public API with host buffers: ingest the couplings
    # from host memory, solve, read back the best spins and the result, every step.
    e2e_t, e2e_u = 0.0, 0
    e2e_steps = args.steps if wl.name == "ea2d" else 1
    for k in range(e2e_steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        i2 = wl.add(ctx)
        if shape is not None:
            ctx.set_shape(i2, **shape)
        r2 = wl.solve(ctx, i2, k)
        ctx.free(i2)
        e2e_t += time.perf_counter() - t
        e2e_u += r2.spin_updates
    n = info["n"]
    h2d = int(info["device_bytes"]) + 4 * wl.R
    d2h = n + 64 + 4 * wl.R + 4

    peaks = load_peaks()
    sm_clock_ghz = (clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0) / 1e3
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    d_mean = statistics.mean(descent_s)
    upd_per_launch = updates / args.steps
    if wl.name == "ea2d":
        # The roofline of the sparse path is HBM: 8 algorithmic bytes per
        # spin-update (the replica's FP32 m read and written once per sweep).
        # This kernel keeps every magnetisation and coupling on chip (about
        # 1 MB of DRAM traffic per launch), so it can run above that line; its
        # own limit is instruction issue, and the SFU ceiling for the method's
        # tanh (one ex2 and one rcp per update; a GB300 SM retires 32 ex2 or 16
        # rcp per clock, measured) is given beside it.
        sh = shape or {}
        rt_used = sh.get("sell_rt", -1) if sh.get("sell_rt", -1) > 0 else 2
        nt_used = sh.get("sell_threads", -1) if sh.get("sell_threads", -1) > 0 else 1024
        tab_used = sh.get("sell_smem_table", -1) != 0
        achieved = 8.0 * upd_per_launch / d_mean / 1e9
        sfu_updates_per_clk = 1.0 / (1.0 / 32.0 + 1.0 / 16.0)
        sfu_peak = sms * sfu_updates_per_clk * sm_clock_ghz * 1e9
        # DRAM bytes per launch (read + write) from one ncu capture of the
        # default shape (2 slots, 1024 threads, table in shared memory); null
        # for another shape, whose counters were not taken.
        default_shape = rt_used == 2 and nt_used == 1024 and tab_used
        traffic = 1.0368e6 + 8.448e3 if default_shape else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                    "bytes_per_update": 8.0,
                    "kernel": "sparse_sell_kernel<RT={}, {} threads, halfword couplings{}, degree 4>".format(
                        rt_used, nt_used, " in shared memory" if tab_used else " through L1"),
                    "peak_source": f"hbm copy ({peaks['source']})",
                    "note": {"bound_in_fact": "instruction issue (state on chip)",
                             "sfu_ceiling_updates_per_s": sfu_peak,
                             "sfu_frac": (upd_per_launch / d_mean) / sfu_peak,
                             "sfu_source": f"{sms} SMs x (1/32 + 1/16 SFU clocks per tanh)^-1 x SM clock"},
                    "descent_ms_mean": 1e3 * d_mean}
    elif wl.name == "ea3d_big":
        # The level launches of one sampled sweep per batch of sweeps (CUDA
        # events on the library's stream), each moving 12 algorithmic bytes
        # per spin-update of its live replicas.
        sh = shape or {}
        rt_used = sh.get("sell_rt", -1) if sh.get("sell_rt", -1) > 0 else 4
        achieved = EA3_BYTES_PER_UPDATE * level_upd / level_s / 1e9 if level_s > 0 else 0.0
        # DRAM bytes per launch: one ncu capture of the staged kernel at RT=4
        # (3.328 GB for a launch of 510 live replicas x 500,000 spins, 13.05 B
        # per live update) scaled by the live updates of a sampled launch;
        # null for another slot width, whose counters were not taken.
        upd_launch = level_upd / level_launches if level_launches else 0.0
        traffic = EA3_DRAM_BYTES_PER_UPDATE * upd_launch if rt_used == 4 else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                    "kernel": f"wide_level_staged_kernel<RT={rt_used}, degree 6> (+-1 words)",
                    "bytes_per_update": EA3_BYTES_PER_UPDATE,
                    "level_launches_sampled": level_launches,
                    "whole_descent_gbs": EA3_BYTES_PER_UPDATE * upd_per_launch / d_mean / 1e9,
                    "peak_source": f"hbm copy ({peaks['source']})",
                    "descent_ms_mean": 1e3 * d_mean}
    else:
        achieved = gemm_flops / gemm_s / 1e12 if gemm_s > 0 else 0.0
        fp8 = wl.precision == "fp8"
        sh = shape or {}
        paired = sh.get("tc_pair", -1) == 1 or (sh.get("tc_pair", -1) == -1 and wl.R >= 2048)
        # an E4M3 contraction's peak: the measured BF16 peak times the nominal
        # FP8 / BF16 ratio (4.5 / 2.25 PFLOP/s dense)
        peak = peaks["bf16_tflops_sustained"] * (2.0 if fp8 else 1.0)
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "{}<128, {}> (tcgen05 {}, split-K)".format(
                        "pair_gemm_kernel" if paired else "panel_gemm_kernel", "FP8" if fp8 else "BF16",
                        "kind::f8f6f4 E4M3" if fp8 else "kind::f16 BF16"),
                    "peak_source": ("2 x bf16 sustained" if fp8 else "bf16 sustained") + f" ({peaks['source']})",
                    "gemm_launches_sampled": gemm_launches,
                    "descent_ms_mean": 1e3 * d_mean}

    vs_fp32 = None
    if rank == 0 and wl.name == "sk8192" and not args.no_fp32_comparison and not args.fixed_sweeps:
        vs_fp32 = fp32_path_comparison(ctx)

    if rank == 0:
        line = {
            "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": wl.dtype,
            "data": "synthetic (seeded instance, Philox start states on device)",
            "config": dict(wl.config, l2="flushed between steps (256 MB write)",
                           parallelism=f"replicas x{world}" if world > 1 else "1 GPU"),
            "e2e": {"value": e2e_u / e2e_t, "unit": "spin-updates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": base,
            "clocks": clocks,
            "best_energy_per_step": best,
        }
        if vs_fp32 is not None:
            line["vs_fp32_path"] = vs_fp32
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_serve(args, world, rank, local):
    """Serving: Poisson arrivals of mixed Ising / max-cut requests, p50/p99 latency.

    The serving configuration's mix: dense SK instances (N 256-16384, +-1 or
    Gaussian couplings) and sparse lattices and random graphs (N 1k-100k,
    degree 4-40), each request asking R replicas in {64, ..., 4096}, under a
    120 GB HBM budget. Two choices keep a 2,000-request run within about a
    quarter of an hour, and the JSON line states both: dense requests take
    at most 64 temperature levels (C_step = T_max / min(2 sqrt(N), 64); the
    paper's 1/sqrt(N) step gives 256 levels at N = 16384), and R is capped by
    size for dense instances (4096 up to N = 1024, 1024 at N = 4096, 256 at
    N = 16384). Dense Gaussian requests and +-1 requests up to N = 1024 run
    on BF16 tensor cores, larger +-1 ones on E4M3 (N = 256: the FP32 path).
    """
    import numpy as np
    import torch

    from paper_1907_05124_gb300 import build, instances, mars
    if rank != 0:
        return
    torch.cuda.set_device(local)
    build.build()
    rng = np.random.default_rng(0)
    ctx = mars.Context(local, hbm_budget_bytes=120 << 30)
    reps_all = np.array([64, 128, 256, 512, 1024, 2048, 4096])
    # (name, inst, n, t_max, c_step, precision, weight, largest R)
    pool = []
    dense_w = {256: 0.10, 1024: 0.06, 4096: 0.03, 16384: 0.005}
    dense_rmax = {256: 4096, 1024: 4096, 4096: 1024, 16384: 256}
    for nn, wgt in dense_w.items():
        lv = min(2.0 * nn ** 0.5, 64.0)
        t_pm1, t_g = 2.0 * nn ** 0.5, 2.0
        pool.append((f"sk_pm1_{nn}", ctx.add_dense(instances.sk_pm1(nn, nn)), nn, t_pm1, t_pm1 / lv,
                     "fp32" if nn == 256 else "bf16" if nn <= 1024 else "fp8", wgt / 2, dense_rmax[nn]))
        pool.append((f"sk_gauss_{nn}", ctx.add_dense(instances.sk_gauss(nn, nn + 1)), nn, t_g, t_g / lv,
                     "fp32" if nn == 256 else "bf16", wgt / 2, dense_rmax[nn]))
    sparse = []
    for L in (32, 64, 100, 200):
        g = instances.ea_lattice(L, 2, L)
        sparse.append((f"ea2d_{L}", ctx.add_csr(*g), g.n, 4.0, 1.0, "fp32"))
    for L in (16, 32):
        g = instances.ea_lattice(L, 3, L)
        sparse.append((f"ea3d_{L}", ctx.add_csr(*g), g.n, 6.0, 1.0, "fp32"))
    for nn, d in ((1000, 40), (5000, 12), (20000, 4), (100000, 4)):
        g = instances.er_graph(nn, d, nn + d, "pm1")
        sparse.append((f"er_{nn}_{d}", ctx.add_csr(*g), g.n, 2.0 * d ** 0.5 + 1.0, 1.0, "fp32"))
    w_sparse = (1.0 - sum(dense_w.values())) / len(sparse)
    pool += [k + (w_sparse, 4096) for k in sparse]
    weights = np.array([k[6] for k in pool])
    n_req = args.requests
    kinds = rng.choice(len(pool), size=n_req, p=weights / weights.sum())
    reps = np.array([rng.choice(reps_all[reps_all <= pool[k][7]]) for k in kinds])
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=n_req))
    ctx.serve_limits(args.inflight)
    pending, lat, upd = {}, [], 0
    by_kind = {}  # request kind -> latencies (s)
    t_start = time.perf_counter()
    nxt = 0
    cancelled = []
    while nxt < n_req or pending:
        now = time.perf_counter() - t_start
        if now > args.serve_deadline:
            for req, (t_arr, name) in list(pending.items()):
                ctx.cancel(req)
                cancelled.append(name)
            for req in list(pending):
                while True:
                    try:
                        if ctx.poll(req) is not None:
                            break
                    except mars.MarsError:
                        break
                    time.sleep(0.001)
            pending.clear()
            break
        while nxt < n_req and arrivals[nxt] <= now:
            name, inst, nn, tmax, cstep, prec = pool[kinds[nxt]][:6]
            req = ctx.submit(inst, int(reps[nxt]), 0.0, tmax, c_step=cstep, seed=nxt,
                             precision=prec)
            pending[req] = (arrivals[nxt], name)
            nxt += 1
        for req in list(pending):
            r = ctx.poll(req)
            if r is not None:
                t_arr, name = pending.pop(req)
                lat.append(time.perf_counter() - t_start - t_arr)
                by_kind.setdefault(name, []).append(lat[-1])
                upd += r.spin_updates
        time.sleep(0.0002)
    wall = time.perf_counter() - t_start
    lat_ms = 1e3 * np.array(lat)
    line = {
        "metric": "spin-updates/s", "value": upd / wall, "unit": "spin-updates/s", "n_gpus": 1,
        "steps": 1, "warmup": 0, "ms_per_step": 1e3 * wall, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16",
        "data": "synthetic (seeded instances, Poisson arrivals)",
        "config": {"workload": f"serving: {n_req} Poisson arrivals at {args.rate}/s, mixed dense SK "
                               "(N 256-16384, +-1 / Gaussian) and sparse lattices / ER graphs "
                               f"(N 1k-100k, degree 4-40), R 64-4096, {args.inflight} in flight, "
                               "120 GB budget",
                   "requests": n_req, "rate_per_s": args.rate, "inflight": args.inflight,
                   "dense_levels": "at most 64 (C_step = T_max / min(2 sqrt(N), 64))",
                   "dense_r_max": {str(k): v for k, v in dense_rmax.items()},
                   "kinds": {k[0]: {"n": k[2], "precision": k[5], "share": round(float(k[6]), 4)}
                             for k in pool}},
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)),
                       "p99": float(np.percentile(lat_ms, 99)),
                       "mean": float(lat_ms.mean()), "max": float(lat_ms.max())},
        "served_by": dict(zip(("persistent_ring_kernel", "own_stream"), ctx.serve_counters())),
        "completed": len(lat), "cancelled_at_deadline": len(cancelled),
        "not_submitted": n_req - nxt,
        "latency_ms_by_kind": {k: {"count": len(v), "p50": float(np.percentile(1e3 * np.array(v), 50)),
                                   "p99": float(np.percentile(1e3 * np.array(v), 99))}
                               for k, v in sorted(by_kind.items())},
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def batch_jobs(instances):
    """The batched configuration: 8 Erdos-Renyi graphs (N in {800, 2000, 5000,
    10000} x mean degree {6, 40}; weights {+1} for the first four, {-1,+1} for
    the rest; seeds 0-7) and a periodic 3-D +-J lattice L=32 (N=32768, seed 8),
    with uneven replica counts between 512 and 4096. T_max is each instance's
    paramagnetic instability scale: about d+1 for {+1} weights (the adjacency's
    top eigenvalue), 2 sqrt(d)+1 for +-1 weights, 6 for the 3-D lattice."""
    graphs, k = [], 0
    for nn in (800, 2000, 5000, 10000):
        for d in (6, 40):
            w = "one" if k < 4 else "pm1"
            tmax = d + 1.0 if w == "one" else 2.0 * d ** 0.5 + 1.0
            graphs.append((f"er_{nn}_{d}_{w}", instances.er_graph(nn, d, k, w), tmax))
            k += 1
    graphs.append(("ea3d_32", instances.ea_lattice(32, 3, 8), 6.0))
    reps = [512, 4096, 1024, 2048, 512, 4096, 1024, 2048, 2048]
    return graphs, reps


def run_batch(args, world, rank, local):
    """One mars_solve_batch over the batched configuration per step: uneven
    instances and replica counts in one persistent launch."""
    import numpy as np
    import torch

    from paper_1907_05124_gb300 import build, instances, mars
    if rank != 0:
        return
    torch.cuda.set_device(local)
    build.build()
    graphs, reps = batch_jobs(instances)
    base = None
    if not args.no_cpu_baseline:
        import oracle as O
        cores = os.cpu_count() or 1
        t_used, upd = 0.0, 0
        for (name, g, tmax), R in zip(graphs, reps):
            m0, t0 = O.draw_replicas(0, cores, g.n, T_MIN, tmax)
            t = time.perf_counter()
            out = O.mars_solve(O.Instance.csr(g), m0, t0, c_step=1.0, d_min=D_MIN, k_max=K_MAX,
                               order=instances.greedy_colour_order(g), nthreads=cores, want_m=False)
            t_used += time.perf_counter() - t
            upd += int(out["sweeps"].sum()) * g.n
        base = {"value": upd / t_used, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{cores} replicas of each of the 9 instances, FP64 oracle, OpenMP over "
                          f"replicas, {t_used:.1f} s"}
    ctx = mars.Context(local)
    insts = [ctx.add_csr(*g) for _, g, _ in graphs]

    def jobs(seed):
        return [(i, R, T_MIN, tmax, {"c_step": 1.0, "d_min": D_MIN, "k_max": K_MAX, "seed": seed + j})
                for j, (i, R, (_, _, tmax)) in enumerate(zip(insts, reps, graphs))]

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = ctx.torch_stream
    for w in range(max(args.warmup, 0)):
        ctx.solve_batch(jobs(10_000 + 100 * w))
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    step_ms, updates, descent_s, launches = [], 0, [], 0
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = ctx.solve_batch(jobs(100 * k))
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        updates += sum(r.spin_updates for r in out)
        descent_s.append(out[0].descent_seconds)
        launches += out[0].kernel_launches
    clocks = sampler.stop()
    tot_ms = sum(step_ms)
    # end to end: ingest every instance from host memory, batch-solve, read back
    torch.cuda.synchronize()
    t = time.perf_counter()
    e2e_ins = [ctx.add_csr(*g) for _, g, _ in graphs]
    saved, insts[:] = list(insts), e2e_ins
    out = ctx.solve_batch(jobs(7))
    for i in e2e_ins:
        ctx.free(i)
    e2e_t = time.perf_counter() - t
    insts[:] = saved
    e2e_u = sum(r.spin_updates for r in out)
    h2d = sum(int(g.row_ptr.nbytes + g.col.nbytes + g.val.nbytes) for _, g, _ in graphs)
    d2h = sum(g.n + 64 for _, g, _ in graphs)
    sfu_updates_per_clk = 1.0 / (1.0 / 32.0 + 1.0 / 16.0)
    sm_clock_ghz = (clocks.get("sm_max_mhz") or 2070.0) / 1e3
    achieved = updates / sum(descent_s)
    peak = 152 * sfu_updates_per_clk * sm_clock_ghz * 1e9
    line = {
        "metric": "spin-updates/s", "value": updates / (tot_ms * 1e-3), "unit": "spin-updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded instances, Philox start states on device)",
        "config": {"workload": "batched: 8 Erdos-Renyi graphs (N 800-10000, mean degree 6/40, weights "
                               "+1 or +-1) and a periodic 3-D +-J lattice L=32, R 512-4096 per instance, "
                               "one persistent launch", "instances": [g[0] for g in graphs],
                   "replicas": reps, "c_step": 1.0, "d_min": D_MIN, "k_max": K_MAX,
                   "l2": "flushed between steps (256 MB write)", "parallelism": "1 GPU"},
        "e2e": {"value": e2e_u / e2e_t, "unit": "spin-updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "spin-updates/s (SFU-bound)", "frac": achieved / peak, "traffic": None,
                     "kernel": "sparse_sell_batch_kernel (persistent, jobs in order)",
                     "peak_source": "152 SMs x (1/32 + 1/16 SFU clocks per tanh)^-1 x SM clock",
                     "descent_ms_mean": 1e3 * sum(descent_s) / len(descent_s)},
        "cpu_baseline": base,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def run_sensitivity(args, world, rank, local):
    """The sensitivity study of the paper's Section 4 on synthetic SK: best and
    mean energy and the fraction P of replicas reaching the best, against the
    number of replicas (1e2, 1e3, 1e4; T0 ~ U(0, lambda) with lambda = 2
    sqrt(N/3), the semicircle edge of U(-1,1) couplings) and against the start
    window ([0,10], [10,20], [20,30]; 1e3 replicas). Couplings uniform in
    (-1, 1), N = 500, 1000, 2000, the FP32 path, C_step 1, d_min 1e-4."""
    import numpy as np
    import torch

    from paper_1907_05124_gb300 import build, instances, mars
    if rank != 0:
        return
    torch.cuda.set_device(local)
    build.build()
    ctx = mars.Context(local)
    cells = []
    t_all = time.perf_counter()
    for n in (500, 1000, 2000):
        inst = ctx.add_dense(instances.sk_uniform(n, n))
        lam = 2.0 * (n / 3.0) ** 0.5
        runs = [("replicas", R, 0.0, lam) for R in (100, 1000, 10000)]
        runs += [("window", 1000, lo, hi) for lo, hi in ((0.0, 10.0), (10.0, 20.0), (20.0, 30.0))]
        for kind, R, lo, hi in runs:
            t = time.perf_counter()
            r = ctx.solve(inst, R, lo, hi, c_step=1.0, d_min=D_MIN, k_max=K_MAX, seed=n + R,
                          outputs=("energies",))
            cells.append({"n": n, "study": kind, "replicas": R, "t_window": [lo, hi],
                          "best": r.best_energy, "mean": r.mean_energy, "P": r.hits / R,
                          "levels_mean": r.levels / R, "solve_s": time.perf_counter() - t})
        ctx.free(inst)
    line = {"metric": "sensitivity table (best, mean, P)", "value": None, "unit": None, "n_gpus": 1,
            "higher_is_better": None, "dtype": "f32", "data": "synthetic (seeded SK instances)",
            "config": {"workload": "SK J_ij ~ U(-1,1), N 500/1000/2000; replicas 1e2/1e3/1e4 at "
                                   "T0 ~ U(0, 2 sqrt(N/3)); windows [0,10]/[10,20]/[20,30] at 1e3 "
                                   "replicas; FP32 sequential sweeps, C_step 1"},
            "cells": cells, "wall_s": time.perf_counter() - t_all}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_ttt(args, world, rank, local):
    """Time to target energy of the tensor-core paths against the plain FP32 path.

    Dense SK with +-1 couplings (N=4096, R=512, T0 ~ U(0, 2 sqrt(N)), C_step 1):
    the same replicas (seed) run on the FP32 SIMT path, the BF16 tcgen05 path
    and the FP8 (E4M3) tcgen05 path. The target is the FP32 path's
    10th-percentile replica energy; a path whose fraction p of replicas reach
    it in a solve of T seconds needs T ln(0.01) / ln(1 - p) to reach it with
    probability 0.99 (independent repeats of the solve).
    """
    import numpy as np
    import torch

    from paper_1907_05124_gb300 import build, instances, mars
    torch.cuda.set_device(local)
    build.build()
    n, R = 4096, args.replicas or 512
    ctx = mars.Context(local)
    inst = ctx.add_dense(instances.sk_pm1(n, 0))
    tmax = 2.0 * n ** 0.5
    runs = {}
    for prec in ("fp32", "bf16", "fp8"):
        kw = dict(c_step=1.0, d_min=D_MIN, k_max=K_MAX, seed=1, precision=prec, outputs=("energies",))
        ctx.solve(inst, R, 0.0, tmax, **dict(kw, seed=2, fixed_sweeps=1))  # warm-up (short)
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = ctx.solve(inst, R, 0.0, tmax, **kw)
        runs[prec] = (time.perf_counter() - t, res)
    target = float(np.percentile(runs["fp32"][1].energies, 10))
    paths = {}
    for prec, (sec, res) in runs.items():
        p = float(np.mean(res.energies <= target))
        ttt = sec * np.log(0.01) / np.log1p(-p) if 0 < p < 1 else (sec if p >= 1 else float("inf"))
        paths[prec] = {"solve_s": sec, "p_target": p, "ttt99_s": ttt, "best_energy": res.best_energy,
                       "spin_updates_per_s": res.spin_updates / sec}
    base = paths["fp32"]["ttt99_s"]
    for prec in paths:
        paths[prec]["speedup_vs_fp32"] = base / paths[prec]["ttt99_s"]
    best_tc = min(("bf16", "fp8"), key=lambda k: paths[k]["ttt99_s"])
    line = {
        "metric": "time to target energy (p = 0.99)", "value": paths[best_tc]["ttt99_s"], "unit": "s",
        "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * runs[best_tc][0],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": best_tc,
        "data": "synthetic (seeded instance, Philox start states on device)",
        "config": {"workload": f"dense SK N={n}, J_ij uniform in {{-1,+1}}, R={R}, T0~U(0,2 sqrt(N)), "
                               "C_step=1, d_min=1e-4, k_max=1000; target = FP32 path's "
                               "10th-percentile energy", "n_spins": n, "replicas": R,
                   "target_energy": target},
        "paths": paths,
        "speedup_vs_fp32_at_equal_ttt": paths[best_tc]["speedup_vs_fp32"],
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "serve":
        run_serve(args, world, rank, local)
        return
    if args.workload == "ttt":
        run_ttt(args, world, rank, local)
        return
    if args.workload == "batch":
        run_batch(args, world, rank, local)
        return
    if args.workload == "sensitivity":
        run_sensitivity(args, world, rank, local)
        return
    run_mars(args, world, rank, local)


if __name__ == "__main__":
    main()
