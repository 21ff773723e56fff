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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mars", choices=["mars", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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


def cpu_baseline(target_s: float):
    """The FP64 oracle on the host cores, on a bounded sample of the same workload."""
    import numpy as np

    import oracle as O
    from paper_1907_05124_gb300 import instances as I

    csr = I.ea_lattice(L, 2, 0)
    inst = O.Instance.csr(csr)
    order = I.greedy_colour_order(csr)
    cores = os.cpu_count() or 1
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


def run_mars(args, world, rank, local):
    import numpy as np
    import torch

    from paper_1907_05124_gb300 import build, instances, mars
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(args.cpu_seconds)  # before any GPU work: plain host threads

    csr = instances.ea_lattice(L, 2, 0)
    ctx = mars.Context(local)
    inst = ctx.add_csr(*csr)
    info = ctx.info(inst)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    stream = ctx.torch_stream  # the stream every library call is ordered on

    def solve(seed):
        return ctx.solve(inst, R, T_MIN, T_MAX, c_step=C_STEP, d_min=D_MIN, k_max=K_MAX,
                         seed=seed, stream=rank, outputs=())

    for w in range(max(args.warmup, 0)):
        solve(10_000 + w)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    step_ms, descent_s, updates = [], [], 0
    best = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()  # L2 flush between timed steps, outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = solve(k)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        descent_s.append(res.descent_seconds)
        updates += res.spin_updates
        best.append(res.best_energy)
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

    # End to end through the public API with host buffers: ingest the CSR from
    # host memory, solve, read back the best spins and the result, every step.
    e2e_t, e2e_u = 0.0, 0
    row_ptr, col, val = csr
    for k in range(args.steps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        i2 = ctx.add_csr(row_ptr, col, val)
        r2 = ctx.solve(i2, R, T_MIN, T_MAX, c_step=C_STEP, d_min=D_MIN, k_max=K_MAX, seed=k,
                       stream=rank, outputs=())
        ctx.free(i2)
        e2e_t += time.perf_counter() - t
        e2e_u += r2.spin_updates
    h2d = int(info["device_bytes"]) + 4 * R
    d2h = L * L + 64 + 4 * R + 4

    # Roofline of the descent kernel (the dominant kernel):
    # the path is bound by SM arithmetic and on-chip traffic, not HBM, since a
    # tile's magnetisations stay in shared memory for the whole descent.
    deg = info["nnz"] / info["n"]
    flop_per_update = 2.0 * deg + 2.0
    d_mean = statistics.mean(descent_s)
    upd_per_launch = updates / args.steps
    achieved = flop_per_update * upd_per_launch / d_mean / 1e12
    sm_clock_ghz = (clocks.get("sm_max_mhz") or 2070.0) / 1e3
    peak = 152 * 128 * 2 * sm_clock_ghz / 1e3  # FP32 FMA lanes x 2 flop x clock, TFLOP/s
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "sparse_sell_kernel<RT=2, 1024 threads, +-1 couplings>",
                "descent_ms_mean": 1e3 * d_mean,
                "spin_updates_per_s_descent": upd_per_launch / d_mean}

    if rank == 0:
        line = {
            "metric": "spin-updates/s", "value": value, "unit": "spin-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded lattice, Philox start states on device)",
            "config": dict(WORKLOAD, l2="flushed between steps (256 MB write)",
                           parallelism=f"replicas x{world}" if world > 1 else "1 GPU"),
            "e2e": {"value": e2e_u / e2e_t, "unit": "spin-updates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": 3 * args.steps,
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
