"""The benchmark's reference arm (the CPU oracle's OpenMP build on all host cores) keeps the JSON
contract on the CPU: one line with impl "reference", exactly the requested K timed steps after
W >= 3 warm-up steps, its own cpu_baseline and an e2e entry with no host-device traffic.  The
OpenMP build steps bit for bit like the plain oracle."""
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
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "OpenMP" in d["cpu_baseline"]["sample"]
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_openmp_oracle_steps_like_the_plain_oracle():
    import numpy as np

    import rodgen
    from oracle.oracle import Oracle, build_oracle_omp, omp_threads, using_library
    p = rodgen.perturbed(rodgen.random_packing(n_rods=60, nmin=3, nmax=30, box=0.08, rest_len=2e-3, radius=0.004,
                                               seed=3, allow_overlap=True, speed=0.3), seed=2)
    ref = Oracle(p).step(*p.state(), dt=2e-6, n_steps=5)
    lib = build_oracle_omp()
    assert omp_threads(lib) >= 1
    with using_library(lib):
        got = Oracle(p).step(*p.state(), dt=2e-6, n_steps=5)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
