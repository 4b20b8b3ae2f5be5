// Checks the integer-pipe FP64 <-> FP32 conversions of rod_fp.h against the host compiler's own
// conversions (round to nearest, ties to even) on edge cases and random bit patterns: the
// range-limited forms (`_bits`, with their ok flag) and the full-range forms (`_all`, bit for
// bit on every input but NaN, where both must give a NaN of the same sign), and the flushing
// forms (`_ftz`: bit for bit in the FP32 normal range, signed zero below it, signed infinity
// above it and for NaN in the rounding; FP32 subnormals widen to signed zero).
// Prints "<checked> <mismatches> <not_ok_in_range> <checked_all> <mismatches_all>
// <checked_ftz> <mismatches_ftz>" and exits 0.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>

#include "../../paper_2605_13766_gb300/csrc/rod_fp.h"

static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t next() {  // xorshift64*
  s ^= s >> 12;
  s ^= s << 25;
  s ^= s >> 27;
  return s * 0x2545F4914F6CDD1Dull;
}

int main() {
  long checked = 0, bad = 0, missed = 0, checked_all = 0, bad_all = 0, checked_ftz = 0, bad_ftz = 0;
  auto same = [](uint64_t a, uint64_t b, bool nan_a, bool nan_b, bool sign_a, bool sign_b) {
    return (nan_a || nan_b) ? (nan_a && nan_b && sign_a == sign_b) : a == b;
  };
  auto check_d = [&](double x) {
    bool ok = false;
    const float got = rod::f32_rn_bits(x, ok);
    const float ref = static_cast<float>(x);
    // ok must hold exactly when the rounded result is zero or normal and x is finite, except for
    // values just below the smallest normal that round up to it (reported not ok, by design)
    const double ax = std::fabs(x);
    const bool in_range = std::isfinite(x) && (ax == 0.0 || (ax >= 0x1p-126 && ax < 0x1p128));
    if (ok) {
      ++checked;
      if (rod::fp32_bits(got) != rod::fp32_bits(ref)) ++bad;
    } else if (in_range) {
      ++missed;
    }
    const float all = rod::f32_rn_all(x);
    ++checked_all;
    if (!same(rod::fp32_bits(all), rod::fp32_bits(ref), std::isnan(all), std::isnan(ref), std::signbit(all),
              std::signbit(ref)))
      ++bad_all;
    // the flushing form: the compiler's result wherever |x| is zero or in [2^-126, 2^128)
    const float ftz = rod::f32_rn_ftz(x);
    const uint32_t sgn = std::signbit(x) ? 0x80000000u : 0u;
    uint32_t want;
    if (std::isnan(x) || ax >= 0x1p128) want = sgn | 0x7F800000u;
    else if (ax < 0x1p-126) want = sgn;
    else want = rod::fp32_bits(ref);
    ++checked_ftz;
    if (rod::fp32_bits(ftz) != want) ++bad_ftz;
  };
  auto check_f = [&](float f) {
    bool ok = false;
    const double got = rod::f64_of_f32_bits(f, ok);
    const bool in_range = std::isfinite(f) && (f == 0.0f || std::fabs(f) >= std::numeric_limits<float>::min());
    const double ref = static_cast<double>(f);
    if (ok) {
      ++checked;
      if (rod::fp64_bits(got) != rod::fp64_bits(ref)) ++bad;
    } else if (in_range) {
      ++missed;
    }
    const double all = rod::f64_of_f32_all(f);
    ++checked_all;
    if (!same(rod::fp64_bits(all), rod::fp64_bits(ref), std::isnan(all), std::isnan(ref), std::signbit(all),
              std::signbit(ref)))
      ++bad_all;
    const double ftz = rod::f64_of_f32_ftz(f);
    const bool sub = std::fpclassify(f) == FP_SUBNORMAL;
    ++checked_ftz;
    if (sub ? rod::fp64_bits(ftz) != (std::signbit(f) ? 0x8000000000000000ull : 0ull)
            : !same(rod::fp64_bits(ftz), rod::fp64_bits(ref), std::isnan(ftz), std::isnan(ref), std::signbit(ftz),
                    std::signbit(ref)))
      ++bad_ftz;
  };
  const double edges[] = {0.0, -0.0, 1.0, -1.0, 0x1p-126, -0x1p-126, 0x1p-127, 0x1.fffffep127, 0x1.ffffffp127,
                          0x1.fffffefffffffp127, 0x1p128, 1e300, -1e-300, INFINITY, -INFINITY, NAN,
                          1.0 + 0x1p-24, 1.0 + 0x1p-23 + 0x1p-24, 1.0 + 0x1p-24 + 0x1p-52, 3.0e-39, 1e-45,
                          0x1p-149, 0x1p-150, 0x1.0000000000001p-150, 0x1.8p-149, 0x1.4p-148, 0x1.fffffcp-127,
                          0x1.fffffep-127, 0x1.fffffdp-127, -0x1p-160, 5e-324, 0x1.fffffffffffffp-127};
  for (double x : edges) check_d(x);
  const float fedges[] = {0.0f, -0.0f, 1.0f, std::numeric_limits<float>::min(), std::numeric_limits<float>::max(),
                          std::numeric_limits<float>::denorm_min(), INFINITY, NAN, -3.5f, -INFINITY, 0x1.fffffcp-127f,
                          -0x1p-140f, 0x1p-149f};
  for (float f : fedges) check_f(f);
  for (int i = 0; i < 2000000; ++i) {
    const uint64_t r = next();
    // exponents spread over the whole range, and concentrated around the FP32 range
    uint64_t u = r;
    if (i & 1) {
      const uint64_t e = 840 + (next() % 350);
      u = (r & 0x800FFFFFFFFFFFFFull) | (e << 52);
    }
    if (i % 4 == 2) u = (u & ~0x1FFFFFFFull) | 0x10000000ull;   // exact ties
    double x;
    std::memcpy(&x, &u, sizeof x);
    check_d(x);
    uint32_t v = static_cast<uint32_t>(r >> 17);
    float f;
    std::memcpy(&f, &v, sizeof f);
    check_f(f);
  }
  // every seventh FP32 subnormal with its neighbouring FP64 values and the tie above it
  for (uint32_t v = 0; v < 0x800000u; v += 7) {
    float f;
    std::memcpy(&f, &v, sizeof f);
    check_f(f);
    check_f(-f);
    const double d = static_cast<double>(f);
    check_d(d);
    check_d(std::nextafter(d, 1.0));
    check_d(std::nextafter(d, -1.0));
    check_d(d + 0x1p-150);   // the ties between neighbouring subnormals
  }
  std::printf("%ld %ld %ld %ld %ld %ld %ld\n", checked, bad, missed, checked_all, bad_all, checked_ftz, bad_ftz);
  return 0;
}
