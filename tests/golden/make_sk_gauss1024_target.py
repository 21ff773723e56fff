"""Write the time-to-target energy of the dense SK instance N = 1024 from the
FP64 oracle, with a large budget.

Time to target (the measurement's definition) takes as its target the best
energy the FP64 oracle reaches on the instance with a large budget. This
script runs the oracle alone (Algorithm 1 in FP64, Section 3) on
`instances.sk_gauss(1024, 3)`, J_ij ~ N(0, 1/N), with the schedule the bench
times on that instance (T0 ~ U(0, 2), C_step = 1/sqrt(N), d_min = 1e-4,
k_max = 1000) for 1024 replicas drawn by the oracle's restatement of the
library's counter-based start-state draw (seed 0), four times the replicas of
one timed solve, and stores the best energy with its provenance in
sk_gauss1024_target.json. It calls nothing but oracle/ and the seeded instance
generator.

    python tests/golden/make_sk_gauss1024_target.py [--replicas 1024] [--threads N]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_1907_05124_gb300 import instances  # noqa: E402

N, INSTANCE_SEED, T_MAX, D_MIN, K_MAX = 1024, 3, 2.0, 1e-4, 1000


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--replicas", type=int, default=1024)
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=os.path.join(HERE, "sk_gauss1024_target.json"))
    args = ap.parse_args()
    J = instances.sk_gauss(N, INSTANCE_SEED)
    oi = O.Instance.dense(J)
    m0, t0 = O.draw_replicas(0, args.replicas, N, 0.0, T_MAX)
    t = time.time()
    energies, sweeps = [], 0
    for b in range(0, args.replicas, 64):
        o = O.mars_solve(oi, m0[b:b + 64], t0[b:b + 64], c_step=1.0 / np.sqrt(N), d_min=D_MIN,
                         k_max=K_MAX, nthreads=args.threads, want_m=False)
        energies.append(o["energy"])
        sweeps += int(o["sweeps"].sum())
        print(f"{b + 64} replicas, best so far {min(e.min() for e in energies):.12g}, "
              f"{time.time() - t:.0f} s", flush=True)
    e = np.concatenate(energies)
    best = float(e.min())
    rec = {
        "instance": f"instances.sk_gauss({N}, {INSTANCE_SEED})",
        "schedule": {"t0": f"U(0, {T_MAX})", "c_step": f"1/sqrt({N})", "d_min": D_MIN, "k_max": K_MAX,
                     "update": "sequential (Algorithm 1, Section 3)"},
        "replicas": args.replicas,
        "draw": "oracle.draw_replicas(seed=0)",
        "best_energy": best,
        "best_replica": int(np.argmin(e)),
        "best_replica_t0": float(t0[int(np.argmin(e))]),
        "hits": int(np.sum(e == best)),
        "energy_p10": float(np.percentile(e, 10)),
        "sweeps": sweeps,
        "oracle_seconds": round(time.time() - t, 1),
        "threads": args.threads,
        "source": "FP64 oracle (oracle/), written by tests/golden/make_sk_gauss1024_target.py",
    }
    with open(args.out, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
