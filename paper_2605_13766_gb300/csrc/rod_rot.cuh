// rod_rot.cuh -- the coefficients of the rotation exponential R = exp([p]x) = (1 - b th^2) I +
// a [p]x + b p p^T, a = sin th / th and b = (1 - cos th) / th^2 with th = |p|, as Taylor series in
// th^2 cut per warp from the largest angle (shared by the step kernels, their adjoint and the
// surrogate's kinematic prior).  Internal to librod.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace rod {

// High 32 bits of a non-negative double: x < 2^k exactly when hi_word(x) < hi_word(2^k), so a
// warp-wide integer maximum of these words bounds every lane's argument.
__device__ __forceinline__ unsigned hi_word(double x) { return static_cast<unsigned>(__double2hiint(x)); }
constexpr unsigned kHi2m20 = 0x3EB00000u;  // 2^-20
constexpr unsigned kHi2m10 = 0x3F500000u;  // 2^-10

// Taylor coefficients in th^2 of a = sin(th)/th and b = (1 - cos th)/th^2: (-1)^k / (2k+1)! and
// (-1)^k / (2k+2)!.
namespace {
__constant__ double kRotA[8] = {1.0, -1.0 / 6.0, 1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0, -1.0 / 39916800.0,
                                1.0 / 6227020800.0, -1.0 / 1307674368000.0};
__constant__ double kRotB[8] = {0.5, -1.0 / 24.0, 1.0 / 720.0, -1.0 / 40320.0, 1.0 / 3628800.0, -1.0 / 479001600.0,
                                1.0 / 87178291200.0, -1.0 / 20922789888000.0};
}  // namespace

// The first n terms of both series by Horner's rule.  The trip count is a loop bound, not an
// unrolled chain, so a warp that needs two terms issues two FMAs and no predicated remainder.
__device__ __forceinline__ void rot_series(double th2, int n, double& a, double& b) {
  a = kRotA[n - 1];
  b = kRotB[n - 1];
#pragma unroll 1
  for (int k = n - 2; k >= 0; --k) {
    a = fma(a, th2, kRotA[k]);
    b = fma(b, th2, kRotB[k]);
  }
}

// sin(th)/th and (1 - cos th)/th^2: 8 terms of the series for th^2 <= 1/4 (the dropped terms are
// below 5e-20 relative there); larger angles use sincos.
__device__ __forceinline__ void rot_coeffs_full(double th2, double& a, double& b) {
  if (th2 <= 0.25) {
    rot_series(th2, 8, a, b);
  } else {
    double th = sqrt(th2);
    double s, c, sh;
    sincos(th, &s, &c);
    sh = sin(0.5 * th) / th;
    a = s / th;
    b = 2.0 * sh * sh;
  }
}

// Same coefficients with the series cut to the warp's largest th^2.  a multiplies K = [p]x and
// b multiplies p p^T, of sizes th and th^2, so a term dropped from a costs R at most its size
// times th: below th^2 = 2^-20 two terms (R off by < th^5 / 120 < 2^-56), below 2^-10 four terms
// (< th^9 / 362880 < 2^-63), otherwise the full series.  The choice is uniform across the warp,
// so lanes never diverge on it.
__device__ __forceinline__ void rot_coeffs(double th2, double& a, double& b) {
  const unsigned mx = __reduce_max_sync(__activemask(), hi_word(th2));
  if (mx < kHi2m10) {
    rot_series(th2, mx < kHi2m20 ? 2 : 4, a, b);
  } else {
    rot_coeffs_full(th2, a, b);
  }
}

}  // namespace rod
