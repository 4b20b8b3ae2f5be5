"""The step kernels' integer-pipe FP64 <-> FP32 conversions (paper_2605_13766_gb300/csrc/rod_fp.h)
against the host compiler's conversions: round to nearest with ties to even, bit for bit, on
edge cases (ties, the ends of the FP32 normal range, zero, infinities, NaN) and 4 million random
bit patterns; every value the conversions decline (ok = false) lies outside their stated range,
except values just below the smallest FP32 normal, which they decline by design.  The full-range
forms (f32_rn_all, f64_of_f32_all) agree with the compiler bit for bit on every input, FP32
subnormals (every seventh, with their ties) and overflow included; NaN maps to NaN of the same
sign.  The flushing forms (f32_rn_ftz, f64_of_f32_ftz) agree with the compiler in the FP32 normal
range and give signed zeros below it and signed infinities above it."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_pipe_conversions_match_the_compiler(tmp_path):
    exe = str(tmp_path / "fp_bits_check")
    subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-o", exe,
                    os.path.join(ROOT, "tests", "csrc", "fp_bits_check.cpp")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    checked, bad, missed, checked_all, bad_all, checked_ftz, bad_ftz = (int(v) for v in out)
    assert checked > 2_500_000
    assert bad == 0
    # the full-range forms: every input, subnormals, overflow, infinities and NaN included
    assert checked_all > 8_000_000
    assert bad_all == 0
    # the flushing forms: exact in the FP32 normal range, signed zero / infinity outside it
    assert checked_ftz == checked_all
    assert bad_ftz == 0
    # only values in [2^-127, 2^-126) (about 1 in 330 of the concentrated exponents) may be declined
    assert missed < 0.01 * checked
