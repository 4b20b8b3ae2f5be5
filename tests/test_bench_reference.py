"""The benchmark's reference arm (the CPU oracle) keeps the JSON contract on the CPU: one line
with impl "reference", exactly the requested K timed steps after W >= 3 warm-up steps, its own
cpu_baseline and an e2e entry with no host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "cantilever", "--steps", "4", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 4 and d["warmup"] == 3    # W raised to 3
    assert d["value"] > 0 and d["unit"] == "element-steps/s" and d["higher_is_better"] is True
    assert abs(d["ms_per_step"] - 1e3 * 100 * int(d["cpu_baseline"]["sample"].split()[2]) / d["value"]) \
        <= 1e-6 * d["ms_per_step"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
