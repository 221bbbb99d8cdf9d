"""The benchmark's GPU line carries the fields its contract asks for."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_fields_on_the_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "3", "--warmup", "3",
         "--no-cpu", "--no-serve", "--no-fp64"],
        cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 3 and d["warmup"] >= 3 and d["n_gpus"] == 1
    assert d["gpu_launches"] == 2 * d["steps"]            # sampling + finalize per step
    assert d["config"]["workload"].startswith("gauss03_N4_P1e6")
    r = d["roofline"]
    assert r["bound"] == "issue" and 0 < r["frac"] < 1.2 and r["peak"] > 0
    assert abs(r["achieved"] / r["peak"] - r["frac"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
