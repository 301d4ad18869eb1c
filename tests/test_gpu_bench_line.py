"""The benchmark's own line on the GPU: one JSON line with the keys of the benchmark
contract, the roofline of the sweep, the FP64 oracle timed on all host cores and on
one, and the accuracy report (each estimate's error against the oracle on the same
draws, beside its Monte Carlo standard error).  A short run: 3 timed steps, no other
workloads, no end-to-end job."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_bench_line_carries_roofline_baseline_and_accuracy():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3",
                          "--no-extras", "--no-e2e", "--no-natural"], cwd=ROOT, capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "accuracy",
                "gpu_launches", "clocks"):
        assert key in d, key
    assert d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0 and d["gpu_launches"] > 0
    r = d["roofline"]
    assert r["bound"] == "hbm" and 0 < r["frac"] < 1.5 and r["achieved"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert cb["one_core"]["cores"] == 1 and cb["one_core"]["value"] > 0
    acc = d["accuracy"]
    for part in ("diagonal", "block"):
        a = acc[part]
        # the FP32 / BF16 errors against FP64 on the same draws are far below the MC error
        assert a["max_abs_error"] >= 0 and a["max_error_over_se"] < 0.5, (part, a)
