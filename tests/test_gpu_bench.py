"""The bench's JSON line on a short run of the headline workload (n = 24):
every key of the line's contract is present and consistent with the others
(the CPU baselines, the literal and batched forms are skipped here to keep the
run short; the driver's default run includes them)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_contract():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "4", "--warmup", "3", "--skip-cpu",
           "--skip-batched", "--skip-literal"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    j = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in j, k
    assert j["n_gpus"] == 1 and j["steps"] == 4 and j["warmup"] >= 3
    assert j["higher_is_better"] is True and j["scaling"] == "weak" and j["data"] == "synthetic"
    assert j["config"]["workload"] and j["config"]["n"] == 24
    # value = the iteration's pairs / time per step
    pairs = 2 * 3 ** 24 - 2 ** 24
    assert abs(j["value"] - pairs / (j["ms_per_step"] / 1000.0)) <= 1e-6 * j["value"]
    roof = j["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in roof, k
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) <= 1e-9 * roof["frac"]
    assert 0.0 < roof["frac"] < 1.5
    e2e = j["e2e"]
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in e2e, k
    assert e2e["unit"] == j["unit"] and 0 < e2e["value"] < j["value"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert j["gpu_launches"] > 0
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in j["clocks"], k
    # the certified bound of the run's p lies above its Blahut lower bound
    f = j["forms"]
    assert f["certified_upper_over_n"] * 24 >= f["lower_after_run"] - 1e-9
