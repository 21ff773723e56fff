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


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_time_to_target_arithmetic():
    """The time-to-target summary: the median over seeds counts a seed that
    missed the target as infinitely slow and is reported only when more than
    half the seeds hit; beside it t ln(0.01) / ln(1 - P); the speedup comes
    from the medians when both exist, else from that form."""
    import math
    b = _bench_module()
    secs = [1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0, 9.0, 10.0]
    hit = [True] * 6 + [False] * 4
    s = b.ttt_summary(secs, hit, reached=6, R=256)
    assert s["ttt_median_s"] == 5.5  # sorted 1..6, inf x4: the 5th and 6th
    P = 6 / 2560
    assert s["P"] == P and s["seeds_reaching_target"] == 6
    assert math.isclose(s["ttt99_s"], 5.5 * math.log(0.01) / math.log(1 - P), rel_tol=1e-12)
    half = b.ttt_summary(secs, [True] * 5 + [False] * 5, reached=5, R=256)
    assert half["ttt_median_s"] is None  # the median of five hits and five misses is not finite
    never = b.ttt_summary(secs, [False] * 10, reached=0, R=256)
    assert never["ttt99_s"] == math.inf and never["ttt_median_s"] is None
    always = b.ttt_summary([2.0] * 10, [True] * 10, reached=2560, R=256)
    assert always["ttt99_s"] == 2.0 and always["ttt_median_s"] == 2.0
    fast = b.ttt_summary([0.5] * 10, hit, reached=6, R=256)
    sp = b.ttt_speedup(s, fast)
    assert sp["speedup_at_equal_ttt"] == 5.5 / 0.5 and sp["speedup_from"].startswith("median")
    sp2 = b.ttt_speedup(half, fast)
    assert math.isclose(sp2["speedup_at_equal_ttt"], half["ttt99_s"] / fast["ttt99_s"])
