"""The FP32 cull in front of the FP64 contact test (paper_2605_13766_gb300/csrc/rod_cull.h) is
conservative: on 2 million random segment pairs (coordinates up to 1.2 m, a third of them
nearly parallel, most near the touching distance) it passes every pair whose exact distance
(long double) is below r_a + r_b (+ skin), for both kinds of FP32 proxy the library forms; and
its second bound (the distance of the two lines) rejects part of the far pairs the first bound
passes.  Contact is the paper's rod-rod interaction (Results, "Fibrous granular materials"); a
pair the cull rejected wrongly would lose a contact force, a pair it passes needlessly costs an
FP64 test."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cull_passes_every_touching_pair(tmp_path):
    exe = str(tmp_path / "cull_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-o", exe, os.path.join(ROOT, "tests", "csrc", "cull_check.cpp")],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True)
    pairs, violations, far, far_b1, far_both = (int(v) for v in out.stdout.split())
    assert pairs == 2_000_000
    assert violations == 0, out.stderr
    assert far > 100_000
    assert far_both < far_b1
    assert far_b1 < 0.05 * far
