// rod_fp.h -- FP64 <-> FP32 conversions by bit manipulation (integer pipe).  Internal to librod.
//
// On this part an FP64 -> FP32 or FP32 -> FP64 conversion instruction issues on the FP64 pipe,
// at the rate of an FP64 fused multiply-add, which the step kernels are bound by.  These
// functions do the same conversions with integer operations on the bit patterns.  The `_bits`
// forms cover the numbers whose conversion stays within the FP32 normal range (and zero) and
// report `ok = false` for the rest (the Newton seeds below need that range); the `_ftz` forms
// flush what lies outside it, without a branch; the `_all` forms cover every input (subnormal
// results, overflow, infinities, NaN), so a caller has no
// conversion instruction to fall back to (a fallback branch that short compiles as a predicated
// instruction, which issues on the FP64 pipe for every warp).  Host-compilable, so the
// bit logic is tested on the CPU against the compiler's own conversions.  Device code also gets
// the FP64 reciprocal and reciprocal square root by Newton-Raphson from seeds formed with them.
#pragma once
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define ROD_FP_HD __host__ __device__ __forceinline__
#else
#define ROD_FP_HD inline
#endif

namespace rod {

ROD_FP_HD uint64_t fp64_bits(double x) {
#if defined(__CUDA_ARCH__)
  return static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}

ROD_FP_HD double fp64_from_bits(uint64_t u) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double(static_cast<long long>(u));
#else
  double x;
  std::memcpy(&x, &u, sizeof x);
  return x;
#endif
}

ROD_FP_HD uint32_t fp32_bits(float x) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, sizeof u);
  return u;
#endif
}

ROD_FP_HD float fp32_from_bits(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, sizeof x);
  return x;
#endif
}

// x rounded to the nearest FP32 (ties to even).  Defined (ok = true) for zero and for every x
// whose double exponent lies in the FP32 normal range [2^-126, 2^128) -- a carry out of the
// largest binade gives infinity, as the rounding should; ok = false otherwise (subnormal FP32
// results, infinities, NaN).
ROD_FP_HD float f32_rn_bits(double x, bool& ok) {
  const uint64_t u = fp64_bits(x);
  const uint32_t hi = static_cast<uint32_t>(u >> 32), lo = static_cast<uint32_t>(u);
  const uint32_t e = (hi >> 20) & 0x7FFu;          // biased FP64 exponent
  const uint32_t sign = hi & 0x80000000u;
  if (e - 897u <= 253u) {                          // 897 <= e <= 1150: FP32 exponent 1..254
    const uint32_t m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    uint32_t bits = sign | ((e - 896u) << 23) | m23;
    const uint32_t rest = lo & 0x1FFFFFFFu;        // the 29 mantissa bits dropped
    if (rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u))) ++bits;
    ok = true;
    return fp32_from_bits(bits);
  }
  if ((hi & 0x7FFFFFFFu) == 0u && lo == 0u) {
    ok = true;
    return fp32_from_bits(sign);
  }
  ok = false;
  return 0.0f;
}

// Count of leading zero bits of a nonzero 32-bit word.
ROD_FP_HD int clz32(uint32_t v) {
#if defined(__CUDA_ARCH__)
  return __clz(static_cast<int>(v));
#else
  return __builtin_clz(v);
#endif
}

// x rounded to the nearest FP32, ties to even, for every x: FP32 normal and subnormal results,
// zero, overflow to infinity, infinities, and NaN (a quiet NaN of x's sign that keeps the top
// bits of x's payload).
ROD_FP_HD float f32_rn_all(double x) {
  const uint64_t u = fp64_bits(x);
  const uint32_t hi = static_cast<uint32_t>(u >> 32), lo = static_cast<uint32_t>(u);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  if (e - 897u <= 253u) {                          // an FP32 normal exponent (carry: infinity)
    uint32_t bits = sign | ((e - 896u) << 23) | m23;
    const uint32_t rest = lo & 0x1FFFFFFFu;
    if (rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u))) ++bits;
    return fp32_from_bits(bits);
  }
  if (e == 0x7FFu) {                               // infinity or NaN
    const bool nan = ((hi & 0xFFFFFu) | lo) != 0u;
    return fp32_from_bits(sign | 0x7F800000u | (nan ? (0x400000u | m23) : 0u));
  }
  if (e > 1150u) return fp32_from_bits(sign | 0x7F800000u);   // |x| >= 2^128
  if (e < 873u) return fp32_from_bits(sign);       // |x| <= 2^-150 (a tie there goes to zero)
  // FP32 subnormal range: |x| = m53 2^(e - 1075) = (m53 2^(e - 926)) units of 2^-149
  const uint64_t m53 = (static_cast<uint64_t>((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
  const uint32_t sh = 926u - e;                    // 30..53
  uint64_t q = m53 >> sh;
  const uint64_t rem = m53 & ((1ull << sh) - 1ull), half = 1ull << (sh - 1u);
  if (rem > half || (rem == half && (q & 1ull))) ++q;   // may carry to the smallest normal
  return fp32_from_bits(sign | static_cast<uint32_t>(q));
}

// An FP32 value widened to FP64 exactly, for every input (subnormals normalised; infinities;
// NaN keeps its payload).
ROD_FP_HD double f64_of_f32_all(float f) {
  const uint32_t b = fp32_bits(f);
  const uint32_t e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  const uint64_t sign = static_cast<uint64_t>(b & 0x80000000u) << 32;
  if (e - 1u <= 253u) return fp64_from_bits(sign | (static_cast<uint64_t>(e + 896u) << 52) | (static_cast<uint64_t>(m) << 29));
  if (e == 0xFFu) return fp64_from_bits(sign | (0x7FFull << 52) | (static_cast<uint64_t>(m) << 29));
  if (m == 0u) return fp64_from_bits(sign);
  const int p = 31 - clz32(m);                     // m 2^-149 = 2^(p - 149) (m / 2^p)
  const uint64_t frac = (static_cast<uint64_t>(m) << (52 - p)) & 0xFFFFFFFFFFFFFull;
  return fp64_from_bits(sign | (static_cast<uint64_t>(p + 874) << 52) | frac);
}

// x rounded to the nearest FP32 (ties to even) when |x| lies in the FP32 normal range or is zero;
// smaller magnitudes give a zero of x's sign, larger ones (and infinities, NaN) an infinity of
// x's sign.  Branch-free integer operations, for code where neither those edge ranges nor a
// conversion instruction are wanted.
ROD_FP_HD float f32_rn_ftz(double x) {
  const uint64_t u = fp64_bits(x);
  const uint32_t hi = static_cast<uint32_t>(u >> 32), lo = static_cast<uint32_t>(u);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const uint32_t sign = hi & 0x80000000u;
  uint32_t bits = sign | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1FFFFFFFu;
  bits += (rest > 0x10000000u || (rest == 0x10000000u && (bits & 1u))) ? 1u : 0u;
  bits = e < 897u ? sign : bits;
  bits = e > 1150u ? (sign | 0x7F800000u) : bits;
  return fp32_from_bits(bits);
}

// An FP32 value widened to FP64 exactly, except that FP32 subnormals give a zero of their sign;
// infinities and NaN (with its payload) carry over.  Branch-free integer operations.
ROD_FP_HD double f64_of_f32_ftz(float f) {
  const uint32_t b = fp32_bits(f);
  const uint32_t e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  const uint32_t sign = b & 0x80000000u;
  uint32_t hi = sign | ((e + 896u) << 20) | (m >> 3);
  uint32_t lo = m << 29;
  hi = e == 0xFFu ? (sign | 0x7FF00000u | (m >> 3)) : hi;
  hi = e == 0u ? sign : hi;
  lo = e == 0u ? 0u : lo;
  return fp64_from_bits((static_cast<uint64_t>(hi) << 32) | lo);
}

// An FP32 value widened to FP64 exactly, for zero and FP32 normal numbers (ok = false for
// subnormals, infinities and NaN).
ROD_FP_HD double f64_of_f32_bits(float f, bool& ok) {
  const uint32_t b = fp32_bits(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint64_t sign = static_cast<uint64_t>(b & 0x80000000u) << 32;
  if (e - 1u <= 253u) {
    const uint64_t m = b & 0x7FFFFFu;
    ok = true;
    return fp64_from_bits(sign | (static_cast<uint64_t>(e + 896u) << 52) | (m << 29));
  }
  ok = (b & 0x7FFFFFFFu) == 0u;
  return fp64_from_bits(sign);
}

#if defined(__CUDACC__)

// 1/x by Newton-Raphson, y <- y + y (1 - x y), from a seed that costs no FP64 instruction: x
// rounded to FP32 on the integer pipe, its correctly rounded FP32 reciprocal, widened on the
// integer pipe (relative error below 2^-23).  Two steps square the error twice, to below the
// FP64 rounding: 4 FP64 instructions.  x whose FP32 rounding or reciprocal leaves the FP32
// normal range takes the FP64 reciprocal instruction sequence instead.
__device__ __forceinline__ double rcp_nr(double x) {
  bool ok1, ok2;
  const float xf = f32_rn_bits(x, ok1);
  const double y0 = f64_of_f32_bits(__frcp_rn(xf), ok2);
  if (!(ok1 && ok2) || xf == 0.0f) return __drcp_rn(x);
  const double e0 = fma(-x, y0, 1.0);
  const double y1 = fma(y0, e0, y0);
  const double e1 = fma(-x, y1, 1.0);
  return fma(y1, e1, y1);
}

// 1/sqrt(x) for x > 0 by one Newton-Raphson step, y <- y + (y/2)(1 - x y^2), from the seed of
// rcp_nr's kind (the correctly rounded FP32 rsqrt of x rounded to FP32: relative error below
// 1.5 2^-24; y/2 formed in FP32 and widened, exactly).  The step leaves a relative error below
// 1.5 (1.5 2^-24)^2 + 2^-52 < 1.3e-14: 3 FP64 instructions.  Otherwise the FP64 rsqrt.
__device__ __forceinline__ double rsqrt_nr(double x) {
  bool ok1, ok2, ok3;
  const float xf = f32_rn_bits(x, ok1);
  const float yf = __frsqrt_rn(xf);
  const double y0 = f64_of_f32_bits(yf, ok2);
  const double h0 = f64_of_f32_bits(0.5f * yf, ok3);
  if (!(ok1 && ok2 && ok3) || !(xf > 0.0f)) return rsqrt(x);
  const double t = x * y0;
  const double r = fma(-t, y0, 1.0);
  return fma(h0, r, y0);
}

// A double rounded to FP32 and an FP32 value widened to FP64 for the surrogate's features and
// update: the branch-free forms (magnitudes outside the FP32 normal range flushed, see above).
// A form with the conversion instruction as the fallback for those ranges compiles to a
// predicated instruction that issues on the FP64 pipe for every warp, and the full-range
// integer forms cost more integer work than that slot saves on the surrogate's latency-bound
// path; the step kernels round with f32_rn_all.
__device__ __forceinline__ float f32_rn(double x) { return f32_rn_ftz(x); }
__device__ __forceinline__ double f64_of(float f) { return f64_of_f32_ftz(f); }

#endif  // __CUDACC__

}  // namespace rod
