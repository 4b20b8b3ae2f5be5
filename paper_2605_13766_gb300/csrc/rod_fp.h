// rod_fp.h -- FP64 <-> FP32 conversions by bit manipulation (integer pipe).  Internal to librod.
//
// On this part an FP64 -> FP32 or FP32 -> FP64 conversion instruction issues on the FP64 pipe,
// at the rate of an FP64 fused multiply-add, which the step kernels are bound by.  These
// functions do the same conversions with integer operations on the bit patterns, for the
// numbers whose conversion stays within the FP32 normal range (and zero); for the rest they
// report `ok = false` and the caller takes the conversion instruction.  Host-compilable, so the
// bit logic is tested on the CPU against the compiler's own conversions.
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

}  // namespace rod
