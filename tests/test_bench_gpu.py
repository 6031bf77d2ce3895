"""bench.py's JSON line on the GPU, on a small case: every key of the contract,
a roofline object, the oracle baseline, the end-to-end number with its byte
counts, launch count and sampled clocks."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_carries_the_contract():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--scale", "14",
                        "--steps", "5", "--warmup", "3", "--cpu-seconds", "0.5",
                        "--e2e-steps", "3"], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 5 and d["warmup"] == 3 and d["n_gpus"] == 1
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] > 0
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert e["value"] < d["value"]       # copies inside the timed region cost time
    assert d["gpu_launches"] == 10     # per step: the product and the split-row sum
    assert d["config"]["workload"] == "rmat-s14-ef16-n128-fp32-grid16x4"
