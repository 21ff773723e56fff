#!/usr/bin/env python
"""MARS benchmark: spin-updates/s on a 2-D Edwards-Anderson +-J spin glass.

Workload (one step): a periodic 100x100 square lattice (N = 10,000 spins,
4 neighbours, J uniform in {-1,+1}, h = 0, seed 0), R = 1024 replicas with
start states and start temperatures T0 ~ U(0, 4) drawn on the device, linear
cooling C_step = 1, d_min = 1e-4, k_max = 1000, sequential sweeps in the
greedy colour order, FP32 local fields; then sign-rounding, exact integer
energies and the best replica. One step is one whole mars_solve.

A spin-update is one new s_i of one replica in one sweep; the metric counts
only the sweeps replicas actually perform.

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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mars", choices=["mars", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="ea2d", choices=["ea2d", "sk8192"],
                    help="ea2d: the 2-D lattice (default); sk8192: dense SK on tensor cores")
    ap.add_argument("--replicas", type=int, default=0, help="override R (profiling runs)")
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


def cpu_baseline(target_s: float, wl=None):
    """The FP64 oracle on the host cores, on a bounded sample of the same workload."""
    import numpy as np

    import oracle as O
    from paper_1907_05124_gb300 import instances as I

    cores = os.cpu_count() or 1
    if wl is not None and wl.name == "sk8192":
        # Dense N=8192 sweeps cost ~0.1 s each on one core: time one sweep per
        # level (fixed-sweep mode) on one replica per core.
        inst = O.Instance.dense(wl.J)
        m0, t0 = O.draw_replicas(0, cores, SK_N, T_MIN, SK_TMAX)
        t = time.perf_counter()
        out = O.mars_solve(inst, m0, t0, c_step=wl.c_step, d_min=D_MIN, k_max=K_MAX,
                           fixed_sweeps=1, nthreads=cores, want_m=False)
        dt = time.perf_counter() - t
        upd = int(out["sweeps"].sum()) * SK_N
        return {"value": upd / dt, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                "sample": f"{cores} replicas of the N=8192 workload, one sweep per level, "
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
    csr = I.ea_lattice(L, 2, 0)
    inst = O.Instance.csr(csr)
    order = I.greedy_colour_order(csr)
    cores = os.cpu_count() or 1
    per_step = cores  # replicas per step: one per host thread

    def step(k):
        m0, t0 = O.draw_replicas(0, per_step, csr.n, T_MIN, T_MAX, r0=(k * per_step) % R)
        t = time.perf_counter()
        out = O.mars_solve(inst, m0, t0, c_step=C_STEP, d_min=D_MIN, k_max=K_MAX, order=order,
                           nthreads=cores, want_m=False)
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
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded lattice, Philox start states)",
        "config": dict(WORKLOAD, sample=f"{per_step} replicas per step"),
        "cpu_baseline": {"value": value, "unit": "spin-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} replicas per step x {args.steps} steps"},
        "e2e": {"value": value, "unit": "spin-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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
        else:
            self.csr = None
            self.J = instances.sk_gauss(SK_N, 0)
            self.R = args.replicas or SK_R
            self.t_max, self.c_step, self.precision = SK_TMAX, 1.0 / SK_N ** 0.5, "bf16"
            self.config = dict(SK_WORKLOAD, replicas=self.R)
            self.dtype = "bf16"
        self.rank = rank

    def add(self, ctx):
        return ctx.add_csr(*self.csr) if self.csr is not None else ctx.add_dense(self.J)

    def solve(self, ctx, inst, seed):
        return ctx.solve(inst, self.R, T_MIN, self.t_max, c_step=self.c_step, d_min=D_MIN,
                         k_max=K_MAX, seed=seed, stream=self.rank, precision=self.precision,
                         outputs=())


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

    for w in range(max(args.warmup, 0)):
        wl.solve(ctx, inst, 10_000 + w)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    step_ms, descent_s, updates, best = [], [], 0, []
    gemm_s, gemm_flops, gemm_launches = 0.0, 0.0, 0
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
    clocks = sampler.stop()
    torch.cuda.synchronize()
    tot_ms = sum(step_ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([tot_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([updates], dtype=torch.float64, device="cuda")
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        tot_ms, updates_all = float(t.item()), float(u.item())
        dist.barrier()
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
        r2 = wl.solve(ctx, i2, k)
        ctx.free(i2)
        e2e_t += time.perf_counter() - t
        e2e_u += r2.spin_updates
    n = info["n"]
    h2d = int(info["device_bytes"]) + 4 * wl.R
    d2h = n + 64 + 4 * wl.R + 4

    peaks = load_peaks()
    sm_clock_ghz = (clocks.get("sm_max_mhz") or 2070.0) / 1e3
    d_mean = statistics.mean(descent_s)
    upd_per_launch = updates / args.steps
    if wl.name == "ea2d":
        # The descent kernel keeps every magnetisation on chip; HBM sees only the
        # coupling table and the outputs. Its ceiling is the SFU: each update
        # needs one exponential and one reciprocal (the tanh), at 16 SFU results
        # per clock per SM.
        sfu_per_update = 2.0
        achieved = sfu_per_update * upd_per_launch / d_mean / 1e12
        peak = 152 * 16 * sm_clock_ghz / 1e3
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T SFU-ops/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "sparse_sell_kernel<RT=2, 1024 threads, +-1 couplings>",
                    "peak_source": "152 SMs x 16 SFU ops/clk x SM clock",
                    "descent_ms_mean": 1e3 * d_mean,
                    "spin_updates_per_s_descent": upd_per_launch / d_mean}
    else:
        achieved = gemm_flops / gemm_s / 1e12 if gemm_s > 0 else 0.0
        peak = peaks["bf16_tflops_sustained"]
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None,
                    "kernel": "panel_gemm_kernel<128> (tcgen05 BF16, split-K)",
                    "peak_source": f"bf16 sustained ({peaks['source']})",
                    "gemm_launches_sampled": gemm_launches,
                    "descent_ms_mean": 1e3 * d_mean}

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
            "gpu_launches": 3 * args.steps if wl.name == "ea2d" else None,
            "roofline": roofline,
            "cpu_baseline": base,
            "clocks": clocks,
            "best_energy_per_step": best,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    run_mars(args, world, rank, local)


if __name__ == "__main__":
    main()
