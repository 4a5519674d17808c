"""The benchmark's contract line on a GPU: one JSON line with the metric,
roofline, clocks, end-to-end and launch-count fields, from a short run."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "5", "--warmup", "3",
                        "--no-cpu-baseline", "--no-batched", "--no-serving"], capture_output=True, text=True,
                       timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "e2e", "gpu_launches"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] == 3 and d["value"] > 0
    # pre-summed series, the pass, the S/N kernel and the detection kernel
    assert d["gpu_launches"] == 4 * 5 and d["config"]["workload"].startswith("apertif")
    rf = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rf, k
    assert rf["bound"] == "alu" and 0 < rf["frac"] < 2 and rf["achieved"] == pytest.approx(rf["frac"] * rf["peak"])
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    t = d["tuning"]  # the stored beam table replayed, its optimum and the default re-timed live
    assert t["ga"]["median_ratio"] <= 1.05 and t["budget"] <= 0.1 * t["valid_points"]
    assert set(t["live_ms"]) == {"optimum", "default"}
