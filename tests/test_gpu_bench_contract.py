"""bench.py's JSON line on a scaled-down workload: one line with the keys the
measurement contract asks for, in consistent units, and a roofline that
divides the dominant family's algorithmic bytes by its measured time."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_keeps_the_contract():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "2", "--warmup", "3",
           "--scale", "0.05", "--no-cpu-baseline", "--no-fp64-path", "--serve-seconds", "0",
           "--no-mixed", "--no-autotune"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
              "gpu_launches", "roofline", "clocks", "fine_level", "per_level", "kernels",
              "measured_peaks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["data"] == "synthetic"
    assert d["value"] > 0 and d["gpu_launches"] > 0
    assert d["e2e"]["unit"] == d["unit"] and d["e2e"]["d2h_bytes_per_step"] > 0
    roof = d["roofline"]
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-3
    assert roof["achieved"] == pytest.approx(
        roof["algorithmic_bytes_per_launch"] / (roof["avg_launch_us"] * 1e3), rel=0.02, abs=0.2)
    assert roof["kernel"] in d["kernels"] and d["kernels"][roof["kernel"]]["bound"] == "hbm"
    # the roofline family is the HBM-bound one with the most device time
    hbm = {k: v["ms"] for k, v in d["kernels"].items() if v["bound"] == "hbm"}
    assert roof["kernel"] == max(hbm, key=hbm.get)
    Ntot = sum(p["N"] for p in d["per_level"])
    assert d["value"] == pytest.approx(Ntot / (d["ms_per_step"] / 1e3), rel=1e-6)
    assert d["fine_level"]["value"] == pytest.approx(
        d["per_level"][-1]["N"] / (d["ms_per_step"] / 1e3), rel=1e-3)
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
