"""CPU check of the bench's reference arm: `bench.py --impl reference` times the FP64 oracle on a
bounded sample of the 640x480 workload and prints one JSON line in the bench's format."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "flows/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    # the line is self-consistent: flows per step over the timed step
    assert abs(d["value"] * d["ms_per_step"] / 1e3 - d["config"]["units_per_step"]) < 1e-6 * d["config"]["units_per_step"]
    assert "102.0 of 409.2" in d["config"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "flows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("640x480")
    assert d["ms_per_step"] > 0 and d["vs_baseline"] is None
