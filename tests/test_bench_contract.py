"""bench.py's command line and the JSON line of its reference arm, on the host.

The reference arm times the FP64 oracle on the host cores (a bounded sample
of the workload per step: by default the dense SK N=8192 workload), so it
runs here without a GPU; its line carries the same keys as the GPU arm's plus
"impl". The workload list is the one the help text and the argument parser
share.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    return out.stdout


@pytest.mark.parametrize("workload,n,R", [(None, 8192, 4096), ("ea2d", 10000, 1024)])
def test_reference_arm_line(workload, n, R):
    extra = ("--workload", workload) if workload else ()
    lines = [ln for ln in run_bench("--impl", "reference", "--steps", "1", "--warmup", "0",
                                    *extra).splitlines()
             if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == "spin-updates/s" and d["unit"] == "spin-updates/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["n_spins"] == n and d["config"]["replicas"] == R
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_workloads_listed():
    text = run_bench("--help", timeout=120)
    for name in ("ea2d", "ea3d_big", "sk8192", "sk8192pm1", "serve", "ttt", "batch", "sensitivity"):
        assert name in text, name
