// rod_cull.h -- the FP32 cull of segment pairs before the FP64 contact test (skin-list build,
// cell search and the listed-pair forces).  Internal to librod; host-compilable so that its
// conservativeness is tested on the CPU against exact segment distances.
//
// A segment is given by its FP32 proxy: midpoint g (xyz) with half length h (w), and half
// edge e (xyz).  The proxies are FP32 roundings of the FP64 segments, within a distance
// tol_p = 1e-6 + 4e-6 (|g_a|_inf + |g_b|_inf + h_a + h_b) of them in the Hausdorff sense (with
// room to spare: the roundings are ~6e-8 |x|), so a lower bound L of the distance of the two
// proxy segments, evaluated with an error below its own margin, gives the FP64 segments a
// distance above L - tol_p.  The cull passes a pair unless one of two lower bounds exceeds
// touch_base + tol_p (touch_base = r_a + r_b, plus the skin when a list is built):
//   1. separation along the axis through the midpoints, dm = g_a - g_b:
//      |dm| - (|e_a . dm| + |e_b . dm|) / |dm|;
//   2. the distance of the two lines, |n . dm| / |n| with n = e_a x e_b, used when the segments
//      are not nearly parallel (|n| >= |e_a| |e_b| / 64, i.e. sin of their angle >= 1/64): the
//      FP32 evaluation of n, n . dm and |n|^2 errs by less than (2 sqrt(3) 64 + 1.25) 2^-22 |dm|
//      < 2^-14 |dm| there; the margin is 2^-12 |dm|.
// Without bound 2, crossed segments a few radii apart passed the cull and took the FP64 test.
#pragma once
#include <cmath>

#if defined(__CUDACC__)
#define ROD_CULL_HD __host__ __device__ __forceinline__
#else
#define ROD_CULL_HD inline
#endif

namespace rod {

#if !defined(__CUDACC__)
struct float4 {
  float x, y, z, w;
};
#endif

ROD_CULL_HD bool may_touch(float4 ga, float4 gb, float4 ea, float4 eb, float touch_base) {
  const float ddx = ga.x - gb.x, ddy = ga.y - gb.y, ddz = ga.z - gb.z;
  const float dm2 = ddx * ddx + ddy * ddy + ddz * ddz;
  const float ma_inf = fmaxf(fabsf(ga.x), fmaxf(fabsf(ga.y), fabsf(ga.z)));
  const float mb_inf = fmaxf(fabsf(gb.x), fmaxf(fabsf(gb.y), fabsf(gb.z)));
  const float touch = touch_base + 1e-6f + 4e-6f * (ma_inf + mb_inf + ga.w + gb.w);
  const float reach = touch + ga.w + gb.w;
  if (dm2 > reach * reach) return false;
  if (!(dm2 > 0.f)) return true;
  const float dm = sqrtf(dm2);
  // 1. separating axis along the midpoints' difference
  const float pa = fabsf(ea.x * ddx + ea.y * ddy + ea.z * ddz);
  const float pb = fabsf(eb.x * ddx + eb.y * ddy + eb.z * ddz);
  if (dm2 - (pa + pb) > touch * dm) return false;
  // 2. distance of the two lines, for segments at least 1/64 rad from parallel
  const float nx = ea.y * eb.z - ea.z * eb.y;
  const float ny = ea.z * eb.x - ea.x * eb.z;
  const float nz = ea.x * eb.y - ea.y * eb.x;
  const float n2 = nx * nx + ny * ny + nz * nz;
  const float ea2 = ea.x * ea.x + ea.y * ea.y + ea.z * ea.z;
  const float eb2 = eb.x * eb.x + eb.y * eb.y + eb.z * eb.z;
  if (4096.f * n2 >= ea2 * eb2) {
    const float pn = nx * ddx + ny * ddy + nz * ddz;
    const float lim = touch + 0x1p-12f * dm;
    if (pn * pn > lim * lim * n2) return false;
  }
  return true;
}

}  // namespace rod
