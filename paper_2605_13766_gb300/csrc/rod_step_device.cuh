// rod_step_device.cuh -- device-side stages of the FP64 rod step shared by the step kernels
// (rod_step.cu) and the adjoint kernel (rod_adjoint.cu), so that the adjoint recomputes the
// forward step with exactly the same arithmetic.  Internal to librod.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "rod_fp.h"
#include "rod_internal.h"
#include "rod_rot.cuh"

namespace rod {
namespace {

// ---------------------------------------------------------------------------------- math

// Exponent field of a double (all ones: Inf or NaN), from its high word on the integer pipe.
__device__ __forceinline__ unsigned exp_field(double x) {
  return static_cast<unsigned>(__double2hiint(x)) & 0x7FF00000u;
}
constexpr unsigned kExpAllOnes = 0x7FF00000u;

// asin(s)/s as a Taylor series in s^2 = |w|^2 (13 terms; dropped tail < 2e-18 for s <= 1/4).
__device__ __forceinline__ double asin_over_s(double s2) {
  double f = 676039.0 / 104857600.0;
  f = fma(f, s2, 88179.0 / 12058624.0);
  f = fma(f, s2, 46189.0 / 5505024.0);
  f = fma(f, s2, 12155.0 / 1245184.0);
  f = fma(f, s2, 6435.0 / 557056.0);
  f = fma(f, s2, 143.0 / 10240.0);
  f = fma(f, s2, 231.0 / 13312.0);
  f = fma(f, s2, 63.0 / 2816.0);
  f = fma(f, s2, 35.0 / 1152.0);
  f = fma(f, s2, 5.0 / 112.0);
  f = fma(f, s2, 3.0 / 40.0);
  f = fma(f, s2, 1.0 / 6.0);
  f = fma(f, s2, 1.0);
  return f;
}

// An FP32 approximation of a double of magnitude at most 2 built from its high word on the
// integer pipe (mantissa cut to 20 bits; magnitudes below 2^-126 give zero); for comparisons
// with wide margins only.
__device__ __forceinline__ float f32_approx_hi(double x) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned sign = hi & 0x80000000u;
  return __uint_as_float(e > 896u ? (sign | ((e - 896u) << 23) | ((hi & 0xFFFFFu) << 3)) : sign);
}

// Coefficients of theta / sin(theta) = asin(s)/s in s^2 (s = sin theta), times 4^-k so that the
// series runs in s4 = 4 s^2: (2k)! / (4^k (k!)^2 (2k+1)) / 4^k.
__constant__ double kTosC[6] = {1.0, 1.0 / 24.0, 3.0 / 640.0, 5.0 / 7168.0, 35.0 / 294912.0, 63.0 / 2883584.0};

// theta / sin(theta) of the relative rotation R = Q_{k+1} Q_k^T, from s4 = |u|^2 = 4 sin^2
// theta (u = (R32 - R23, R13 - R31, R21 - R12)).  Warp-uniform cut of the series like
// rot_coeffs (sin^2 < 2^-20: three terms, dropped < 4e-20; sin^2 < 2^-10: six terms, dropped
// < 2e-20) when every lane's rotation is small.  With sin^2 < 2^-10 the angle is below 1.8 deg
// or above 178.2 deg; above 178.2 deg, dd_a = d_a(k+1) . d_a(k) = cos t + (1 - cos t)(n . d_a)^2
// < 2 (n . d_a)^2 - 0.9995 (n the axis), so dd1 and dd3 cannot both exceed 1/4 (that needs
// (n . d1)^2 + (n . d3)^2 > 1.249), while below 1.8 deg both exceed cos t > 0.9995.  The test
// takes dd1 and dd3 in FP32 from the high words of the directors (integer and FP32 pipes; their
// error, below 1e-5, is far inside the margins); FP64 dot products and cos theta are formed only
// off the fast path.
__device__ __forceinline__ double theta_over_sin(double s4, const double* qa, const double* qb) {
  constexpr unsigned kHi2m18 = 0x3ED00000u;  // 4 x 2^-20
  constexpr unsigned kHi2m8 = 0x3F700000u;   // 4 x 2^-10
  const unsigned act = __activemask();
  const unsigned mx = __reduce_max_sync(act, hi_word(s4));
  float d1 = 0.f, d3 = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    d1 = fmaf(f32_approx_hi(qb[c]), f32_approx_hi(qa[c]), d1);
    d3 = fmaf(f32_approx_hi(qb[6 + c]), f32_approx_hi(qa[6 + c]), d3);
  }
  const bool small = __all_sync(act, d1 > 0.25f && d3 > 0.25f);
  if (small && mx < kHi2m8) {
    // the series in sin^2 = s4 / 4, its coefficients scaled by powers of 1/4, by Horner's rule
    // over a warp-uniform trip count (no predicated remainder)
    int k = (mx < kHi2m18) ? 2 : 5;
    double f = kTosC[k];
#pragma unroll 1
    for (--k; k >= 0; --k) f = fma(f, s4, kTosC[k]);
    return f;
  }
  const double s2 = 0.25 * s4;
  const double dd1 = fma(qb[0], qa[0], fma(qb[1], qa[1], qb[2] * qa[2]));
  const double dd2 = fma(qb[3], qa[3], fma(qb[4], qa[4], qb[5] * qa[5]));
  const double dd3 = fma(qb[6], qa[6], fma(qb[7], qa[7], qb[8] * qa[8]));
  const double c = 0.5 * ((dd1 + dd2 + dd3) - 1.0);
  if (s2 <= 0.0625 && c > 0.0) return asin_over_s(s2);
  const double sn = sqrt(s2);
  return (sn > 0.0) ? atan2(sn, c) / sn : 1.0;
}

struct Smem {
  double *X, *VN, *QQ, *WW;     // state
  double *NF, *TA, *ELL, *EDIL; // element work (EDIL: dilatation over rest length, e / rl)
  double *PP, *TT;              // Voronoi work
  double* ACT;                  // per-rod actuation value (1/rl and 1/m are read through L1)
  double* BF;                   // [4] magnetic field b(t) of the step and its force time t
  int* rel0;                    // [CR+1] first element of each rod (pack-local)
  // per pack-local rod: global rod index, and the offsets from pack-local element / node /
  // Voronoi indices to global ones (global = local + offset)
  int *grod, *dE, *dN, *dV;
  short *erod, *nrod, *vrod;    // pack-local rod of each element / node / Voronoi point
  float* XF;                    // [3][CN] node positions rounded to FP32 by the kinematic stage, or null
  int CE, CN, CV, CR;
  // the threads that share the pack: this thread's index and their number (a block, or the
  // whole grid of a cooperative launch whose working arrays live in global memory)
  int t0, ts;
  bool grid;
};

// Barrier between stages: the block, or the whole grid of a cooperative launch.
__device__ __forceinline__ void stage_sync(const Smem& m) {
  if (m.grid) {
    cooperative_groups::this_grid().sync();
  } else {
    __syncthreads();
  }
}

__device__ __forceinline__ Smem carve(double* base, const LaunchShape& S) {
  Smem m;
  m.CE = S.cap_elems;
  m.CR = S.cap_rods;
  m.CN = m.CE + m.CR;
  m.CV = m.CE;
  double* p = base;
  m.X = p;    p += 3 * m.CN;
  m.VN = p;   p += 3 * m.CN;
  m.QQ = p;   p += 9 * m.CE;
  m.WW = p;   p += 3 * m.CE;
  m.NF = p;   p += 3 * m.CE;
  m.TA = p;   p += 3 * m.CE;
  m.ELL = p;  p += m.CE;
  m.EDIL = p; p += m.CE;
  m.PP = p;   p += 3 * m.CV;
  m.TT = p;   p += 3 * m.CV;
  m.ACT = p;  p += m.CR;
  m.BF = p;   p += 4;
  m.rel0 = reinterpret_cast<int*>(p);
  m.grod = m.rel0 + m.CR + 1;
  m.dE = m.grod + m.CR;
  m.dN = m.dE + m.CR;
  m.dV = m.dN + m.CR;
  m.erod = reinterpret_cast<short*>(m.dV + m.CR);
  m.nrod = m.erod + m.CE;
  m.vrod = m.nrod + m.CN;
  m.XF = nullptr;
  m.t0 = threadIdx.x;
  m.ts = blockDim.x;
  m.grid = false;
  return m;
}

__device__ __forceinline__ int find_rod(const int* starts, int nrods, int idx) {
  // largest r with starts[r] <= idx (starts increasing, starts[0] = 0)
  int lo = 0, hi = nrods - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= idx) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ kinematic stage (a1/a11, a2)

// Kinematic update of one element: Q <- exp(-h [w]x) Q (clamped element: held value).
__device__ __forceinline__ void kin_element(const StepParams& P, const Pack& pk, Smem& m, int i, double h) {
  const int r = m.erod[i];
  const int g = m.grod[r];
  const bool held = (i == m.rel0[r]) && P.rods[g].clamp;
  double q[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) q[a] = m.QQ[a * m.CE + i];
  if (held) {
#pragma unroll
    for (int a = 0; a < 9; ++a) q[a] = P.clamp_Q[a * P.n_rods + g];
  } else {
    // Q <- R Q, R = exp([phi]x), phi = -h w:  R = I + a K + b K^2 = (1 - b th^2) I + a K + b phi phi^T.
    // The directors are the rows of Q: d1' and d2' take rows 0 and 1 of R, and d3' = d1' x d2'
    // (the same rotation of a right-handed orthonormal frame; 6 entries of R instead of 9, and 24
    // products instead of 27).
    const double p0 = -h * m.WW[i], p1 = -h * m.WW[m.CE + i], p2 = -h * m.WW[2 * m.CE + i];
    const double th2 = fma(p0, p0, fma(p1, p1, p2 * p2));
    double ca, cb;
    rot_coeffs(th2, ca, cb);
    const double c0 = fma(-cb, th2, 1.0);
    const double b0 = cb * p0, b1 = cb * p1;
    const double a0 = ca * p0, a1 = ca * p1, a2 = ca * p2;
    const double R00 = fma(b0, p0, c0), R11 = fma(b1, p1, c0);
    const double R01 = fma(b0, p1, -a2), R10 = fma(b1, p0, a2);
    const double R02 = fma(b0, p2, a1), R12 = fma(b1, p2, -a0);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double q0 = q[c], q1 = q[3 + c], q2 = q[6 + c];
      q[c] = fma(R00, q0, fma(R01, q1, R02 * q2));
      q[3 + c] = fma(R10, q0, fma(R11, q1, R12 * q2));
    }
    q[6] = fma(q[1], q[5], -q[2] * q[4]);
    q[7] = fma(q[2], q[3], -q[0] * q[5]);
    q[8] = fma(q[0], q[4], -q[1] * q[3]);
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) m.QQ[a * m.CE + i] = q[a];
}

// Kinematic update of one node: x <- x + h v (clamped node: held value).
__device__ __forceinline__ void kin_node(const StepParams& P, const Pack& pk, Smem& m, int j, double h) {
  const int r = m.nrod[j];
  const int g = m.grod[r];
  const bool held = (j == m.rel0[r] + r) && P.rods[g].clamp;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double val = held ? P.clamp_x[c * P.n_rods + g] : fma(h, m.VN[c * m.CN + j], m.X[c * m.CN + j]);
    m.X[c * m.CN + j] = val;
    if (m.XF) m.XF[c * m.CN + j] = f32_rn_all(val);   // integer pipe for every input
  }
}

__device__ __forceinline__ void kinematic(const StepParams& P, const Pack& pk, Smem& m, double h) {
  const int Ep = pk.nelem, Np = pk.nnode;
  for (int i = m.t0; i < Ep; i += m.ts) kin_element(P, pk, m, i, h);
  for (int j = m.t0; j < Np; j += m.ts) kin_node(P, pk, m, j, h);
}

// --------------------------------------------------------------- dynamic stage (a3-a7, a10, a2)

// Feature sets of the stage functions (template argument FS): a stage compiled for a set tests
// only the features in it, the others being false at compile time, so that none of their
// predicated instructions reaches the FP64 pipe.  FS = 0 is the plain step (circular sections
// without rest strain or curvature, no loads but gravity and contact); kFeatAll tests them all.
constexpr int kFeatRest = 1;   // rest strain or rest curvature
constexpr int kFeatExt = 2;    // element couples, magnetic field, muscles, walls, tip forces
constexpr int kFeatAct = 4;    // actuation couples
constexpr int kFeatDamp = 8;   // linear or rotational damping, drag
constexpr int kFeatAll = 15;

// Stage A (elements): geometry, shear strain, internal force, shear couple, transport couples,
// damping and external couples.
template <int FS = kFeatAll>
__device__ __forceinline__ void stage_elements(const StepParams& P, const Pack& pk, Smem& m) {
  const int Ep = pk.nelem;
  for (int i = m.t0; i < Ep; i += m.ts) {
    const int r = m.erod[i];
    const RodConst* rc = P.rods + m.grod[r];
    const int j = i + r;
    const int ge = i + m.dE[r];
    double l[3], dv[3], q[9], w[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      l[c] = m.X[c * m.CN + j + 1] - m.X[c * m.CN + j];
      dv[c] = m.VN[c * m.CN + j + 1] - m.VN[c * m.CN + j];
      w[c] = m.WW[c * m.CE + i];
    }
#pragma unroll
    for (int a = 0; a < 9; ++a) q[a] = m.QQ[a * m.CE + i];
    const double ll = fma(l[0], l[0], fma(l[1], l[1], l[2] * l[2]));
    const double rs = rsqrt_nr(ll);         // 1 / ell
    const double ell = ll * rs;
    const double rl = __ldg(P.rest_len + ge);
    const double ie = rl * rs;              // 1 / e
    double Ql[3], sg[3], n[3], tc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) Ql[a] = fma(q[3 * a], l[0], fma(q[3 * a + 1], l[1], q[3 * a + 2] * l[2]));
    // n / e = S sigma / e  (the 1/e of the internal force, folded once), and the shear couple
    // ((Q t) x n) rl = (Ql x n) rl / ell = Ql x (n / e)
    if ((FS & kFeatRest) && P.rest_sigma) {
      const double irl = __ldg(P.inv_rl + ge);
      sg[0] = Ql[0] * irl;
      sg[1] = Ql[1] * irl;
      sg[2] = fma(Ql[2], irl, -1.0);
#pragma unroll
      for (int c = 0; c < 3; ++c) sg[c] -= __ldg(P.rest_sigma + c * P.E + ge);
#pragma unroll
      for (int c = 0; c < 3; ++c) n[c] = (__ldg(&rc->S[c]) * ie) * sg[c];
      tc[0] = fma(Ql[1], n[2], -Ql[2] * n[1]);
      tc[1] = fma(Ql[2], n[0], -Ql[0] * n[2]);
      tc[2] = fma(Ql[0], n[1], -Ql[1] * n[0]);
    } else {
      // sigma / e = (Q l / rl - e3) rl / ell = Q l / ell - e3 rl / ell  (S[0] = S[1]), so
      // n_0,1 = s01 Ql_0,1 and Ql x n = (Ql_1 z, -Ql_0 z, 0) with z = n_2 - s01 Ql_2
      const double s2 = __ldg(&rc->S[2]);
      const double s01 = __ldg(&rc->S[0]) * rs;
      n[0] = s01 * Ql[0];
      n[1] = s01 * Ql[1];
      n[2] = s2 * fma(rs, Ql[2], -ie);
      const double z = fma(-s01, Ql[2], n[2]);
      tc[0] = Ql[1] * z;
      tc[1] = -Ql[0] * z;
      tc[2] = 0.0;
    }
    // lab internal force N = Q^T n / e
#pragma unroll
    for (int b = 0; b < 3; ++b) m.NF[b * m.CE + i] = fma(q[b], n[0], fma(q[3 + b], n[1], q[6 + b] * n[2]));
    // transport couples (J w / e) x w + (J w / e^2) de/dt,  de/dt = (l . dv) / (ell rl), and the
    // rotational damping -nu rl (I/A) w; with J w = rl g, g = rho I w:
    //   rl/e (g x w) + rl (de/dt / e^2 - damp_rot) g
    // For a circular section rho I = (j, j, j3): g x w = (j - j3)(w1 w2, -w0 w2, 0).
    // rl (de/dt / e^2 - damp_rot) = ie^2 ((l . dv) rs) - rl damp_rot   (rl / (ell rl e^2) = ie^2 rs)
    const double ldv = fma(l[0], dv[0], fma(l[1], dv[1], l[2] * dv[2]));
    const double k1 = (rl * ie) * __ldg(&rc->rhoI_12);
    const double k2 = ((FS & kFeatDamp) && P.has_damp_rot) ? fma(ie * ie, ldv * rs, -rl * __ldg(&rc->damp_rot)) : (ie * ie) * (ldv * rs);
    tc[0] = fma(k1, w[1] * w[2], tc[0]);
    tc[1] = fma(-k1, w[0] * w[2], tc[1]);
    const double k2j = k2 * __ldg(&rc->rhoI[0]);
    tc[0] = fma(k2j, w[0], tc[0]);
    tc[1] = fma(k2j, w[1], tc[1]);
    tc[2] = fma(k2 * __ldg(&rc->rhoI[2]), w[2], tc[2]);
    if ((FS & kFeatExt) && P.elem_couple) {
#pragma unroll
      for (int c = 0; c < 3; ++c) tc[c] += __ldg(P.elem_couple + c * P.E + ge);
    }
    if ((FS & kFeatAct) && P.has_act && (i - m.rel0[r]) == rc->act_elem) tc[0] += m.ACT[r];
    if ((FS & kFeatExt) && P.magnet) {
      // magnetic couple rl (m x (Q b)), Q b: the field in the element's frame
      double qb[3], mg[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) qb[a] = fma(q[3 * a], m.BF[0], fma(q[3 * a + 1], m.BF[1], q[3 * a + 2] * m.BF[2]));
#pragma unroll
      for (int c = 0; c < 3; ++c) mg[c] = rl * __ldg(P.magnet + c * P.E + ge);
      tc[0] += fma(mg[1], qb[2], -mg[2] * qb[1]);
      tc[1] += fma(mg[2], qb[0], -mg[0] * qb[2]);
      tc[2] += fma(mg[0], qb[1], -mg[1] * qb[0]);
    }
    if ((FS & kFeatExt) && P.arc0 && rc->muscle_amp != 0.0) {
      // muscle couples about d1 at the Voronoi points on both sides: tau_{i-1} - tau_i
      const int li = i - m.rel0[r], nr = m.rel0[r + 1] - m.rel0[r];
      const double t = m.BF[3], sl = __ldg(P.arc0 + ge), sr = sl + rl;
      const double tr = (li <= nr - 2) ? rc->muscle_amp * sin(rc->muscle_omega * t - rc->muscle_k * sr + rc->muscle_phase) : 0.0;
      const double tl = (li >= 1) ? rc->muscle_amp * sin(rc->muscle_omega * t - rc->muscle_k * sl + rc->muscle_phase) : 0.0;
      tc[0] += tl - tr;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) m.TA[c * m.CE + i] = tc[c];
    m.ELL[i] = ell;
    m.EDIL[i] = ell * __ldg(P.inv_rl2 + ge);   // e / rl, the factor of the angular acceleration
  }
}

// Stage B (Voronoi points): curvature by the rotation logarithm, Voronoi dilatation,
// bending/twist couple m = B(kappa - kappa0), P = m/eps^3, T = (kappa x m) D/eps^3.  The
// element couple of stage C takes P_k - P_{k-1} + (T_k + T_{k-1}) / 2 over its two Voronoi
// points, so each point stores its two shares: PP = P + T/2 (to the element on its left) and
// TT = T/2 - P (to the element on its right).  For a circular section without rest curvature
// T_3 = 0: PP holds P_3 and TT's third component is not written.
template <int FS = kFeatAll>
__device__ __forceinline__ void stage_voronoi(const StepParams& P, const Pack& pk, Smem& m) {
  const int Vp = pk.nvor;
  for (int k = m.t0; k < Vp; k += m.ts) {
    const int r = m.vrod[k];
    const RodConst* rc = P.rods + m.grod[r];
    const int i = k + r;
    const int gv = k + m.dV[r];
    double qa[9], qb[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      qa[a] = m.QQ[a * m.CE + i];
      qb[a] = m.QQ[a * m.CE + i + 1];
    }
    // R = Q_{k+1} Q_k^T, R_ab = d_a(k+1) . d_b(k);  u = (R32 - R23, R13 - R31, R21 - R12)
    double u0 = qb[6] * qa[3];
    u0 = fma(qb[7], qa[4], u0);
    u0 = fma(qb[8], qa[5], u0);
    u0 = fma(-qb[3], qa[6], u0);
    u0 = fma(-qb[4], qa[7], u0);
    u0 = fma(-qb[5], qa[8], u0);
    double u1 = qb[0] * qa[6];
    u1 = fma(qb[1], qa[7], u1);
    u1 = fma(qb[2], qa[8], u1);
    u1 = fma(-qb[6], qa[0], u1);
    u1 = fma(-qb[7], qa[1], u1);
    u1 = fma(-qb[8], qa[2], u1);
    double u2 = qb[3] * qa[0];
    u2 = fma(qb[4], qa[1], u2);
    u2 = fma(qb[5], qa[2], u2);
    u2 = fma(-qb[0], qa[3], u2);
    u2 = fma(-qb[1], qa[4], u2);
    u2 = fma(-qb[2], qa[5], u2);
    const double s4 = fma(u0, u0, fma(u1, u1, u2 * u2));  // |u|^2 = 4 sin^2(theta)
    const double f = theta_over_sin(s4, qa, qb);
    const double ls = m.ELL[i] + m.ELL[i + 1];   // eps = ls / (2D)
    if ((FS & kFeatRest) && P.rest_kappa) {
      const double i2D = __ldg(P.inv_2D + gv);
      const double ieps = rcp_nr(ls * i2D);
      const double ie3 = ieps * ieps * ieps;
      const double kf = -f * i2D;           // kappa = -(theta/s) w / D = -f u / (2D)
      const double tDh = (0.5 * __ldg(P.Dhat + gv)) * ie3;
      const double kap[3] = {kf * u0, kf * u1, kf * u2};
      double mk[3];
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) mk[cc] = __ldg(&rc->B[cc]) * (kap[cc] - __ldg(P.rest_kappa + cc * P.V + gv));
      const double cr[3] = {fma(kap[1], mk[2], -kap[2] * mk[1]), fma(kap[2], mk[0], -kap[0] * mk[2]),
                            fma(kap[0], mk[1], -kap[1] * mk[0])};
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        const double pc = mk[cc] * ie3;
        m.PP[cc * m.CV + k] = fma(cr[cc], tDh, pc);
        m.TT[cc * m.CV + k] = fma(cr[cc], tDh, -pc);
      }
    } else {
      // m = B kappa = kf B u with kf = -f / (2D); with B = (b, b, b3) (circular section) kappa x m
      // = kf^2 (b3 - b) (u1 u2, -u0 u2, 0), and as D / (2D) = 1/2 exactly, T/2 = kf^2 D / (2 eps^3)
      // (kappa x m) / kf^2 = f g B_21 / 4 (u1 u2, -u0 u2, 0) with g = f / (2D eps^3) = f (2D)^2 / ls^3
      const double is = rcp_nr(ls);
      const double g = (f * (is * is * is)) * __ldg(P.sq_2D + gv);
      const double sb = -g * __ldg(&rc->B[0]);
      const double ct = (f * g) * __ldg(&rc->B_21q);
      const double p0 = sb * u0, p1 = sb * u1;
      const double u12 = u1 * u2, u02 = u0 * u2;
      m.PP[k] = fma(ct, u12, p0);
      m.TT[k] = fma(ct, u12, -p0);
      m.PP[m.CV + k] = fma(-ct, u02, p1);
      m.TT[m.CV + k] = fma(-ct, u02, -p1);
      m.PP[2 * m.CV + k] = (-g * __ldg(&rc->B[2])) * u2;
    }
  }
}

// The element couple of element i from its Voronoi points (right: k, if hasR; left: k - 1, if
// hasL) and its own couple TA: P_k - P_{k-1} + (T_k + T_{k-1}) / 2 + TA as PP_k + TT_{k-1} + TA.
template <int FS = kFeatAll>
__device__ __forceinline__ void element_couple(const StepParams& P, const Smem& m, int i, int k, bool hasR, bool hasL,
                                               double tau[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double Ar = hasR ? m.PP[c * m.CV + k] : 0.0;
    if (c == 2 && !((FS & kFeatRest) && P.rest_kappa)) {
      const double Al = hasL ? m.PP[c * m.CV + k - 1] : 0.0;
      tau[c] = (Ar - Al) + m.TA[c * m.CE + i];
    } else {
      const double Bl = hasL ? m.TT[c * m.CV + k - 1] : 0.0;
      tau[c] = (Ar + Bl) + m.TA[c * m.CE + i];
    }
  }
}

// Stage C (elements): bending couple from the difference and trapezoid operators, angular
// acceleration e J^{-1} tau, rate update and constraint; optional kinematic rotation.
template <int MODE, int FS = kFeatAll>
__device__ __forceinline__ void stage_rotation(const StepParams& P, const Pack& pk, Smem& m, double dt, double h,
                                               double* acc_w) {
  const int Ep = pk.nelem;
  for (int i = m.t0; i < Ep; i += m.ts) {
    const int r = m.erod[i];
    const int g = m.grod[r];
    const int ge = i + m.dE[r];
    const RodConst* rc = P.rods + g;
    const int first = m.rel0[r];
    const int nr = m.rel0[r + 1] - first;
    const int li = i - first;
    const int k = i - r;                     // right Voronoi point (valid if li < nr-1)
    const bool hasR = li < nr - 1, hasL = li > 0;
    double tau[3];
    element_couple<FS>(P, m, i, k, hasR, hasL, tau);
    const bool held = (li == 0) && rc->clamp;
    if (MODE == MODE_RHS) {
      const double ke = m.EDIL[i];
#pragma unroll
      for (int c = 0; c < 3; ++c) acc_w[c * P.E + ge] = held ? 0.0 : ke * __ldg(&rc->inv_rhoI[c]) * tau[c];
    } else {
      // w += dt e J^{-1} tau,  J^{-1} = 1/(rho I rl)  (inv_rhoI[0] = inv_rhoI[1]; EDIL = e / rl)
      const double ke = dt * m.EDIL[i];
      const double k01 = ke * __ldg(&rc->inv_rhoI[0]), k2 = ke * __ldg(&rc->inv_rhoI[2]);
      m.WW[i] = held ? 0.0 : fma(k01, tau[0], m.WW[i]);
      m.WW[m.CE + i] = held ? 0.0 : fma(k01, tau[1], m.WW[m.CE + i]);
      m.WW[2 * m.CE + i] = held ? 0.0 : fma(k2, tau[2], m.WW[2 * m.CE + i]);
      // the following kinematic half/full step of this element (it reads only its own w, Q)
      if (h != 0.0) kin_element(P, pk, m, i, h);
    }
  }
}

// Stage D (nodes): internal force difference, external forces, velocity update + constraint.
template <int MODE, int FS = kFeatAll>
__device__ __forceinline__ void stage_translation(const StepParams& P, const Pack& pk, Smem& m, double dt,
                                                  double* acc_v, double t, double h = 0.0) {
  const int Np = pk.nnode;
  const double dtg[3] = {dt * P.gravity[0], dt * P.gravity[1], dt * P.gravity[2]};
  for (int j = m.t0; j < Np; j += m.ts) {
    const int r = m.nrod[j];
    const int g = m.grod[r];
    const int gn = j + m.dN[r];
    const RodConst* rc = P.rods + g;
    const int firstn = m.rel0[r] + r;
    const int nr = m.rel0[r + 1] - m.rel0[r];
    const int lj = j - firstn;
    const bool hasR = lj < nr, hasL = lj > 0;
    const int iR = j - r;                    // element to the right (pack-local)
    const bool held = (lj == 0) && rc->clamp;
    const double im = __ldg(P.inv_m + gn);
    const double dl = __ldg(&rc->damp_lin);
    double F[3];
    bool contact = false;
    int ge = 0;
    bool fR = false, fL = false;
    if (P.fseg) {
      // contact: node a of segment iR and node b of segment iR-1; with the skin list only
      // segments with candidates have entries (bit set in fmask)
      ge = iR + m.dE[r];
      fR = hasR && (!P.fmask || ((__ldg(P.fmask + (ge >> 5)) >> (ge & 31)) & 1u));
      fL = hasL && (!P.fmask || ((__ldg(P.fmask + ((ge - 1) >> 5)) >> ((ge - 1) & 31)) & 1u));
      // warps without a contact force take the plain difference (the common case)
      contact = __any_sync(__activemask(), fR || fL);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double Nr = hasR ? m.NF[c * m.CE + iR] : 0.0;
      const double Nl = hasL ? m.NF[c * m.CE + iR - 1] : 0.0;
      F[c] = Nr - Nl;
    }
    if (contact) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double fa = fR ? __ldg(P.fseg + c * P.E + ge) : 0.0;
        const double fb = fL ? __ldg(P.fseg + (3 + c) * P.E + ge - 1) : 0.0;
        F[c] += fa + fb;
      }
    }
    if ((FS & kFeatExt) && P.has_tip && lj == nr) {
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c] += __ldg(&rc->tip[c]);
    }
    for (int k = 0; k < ((FS & kFeatExt) ? P.n_walls : 0); ++k) {
      // node sphere (radius of the rod) against the half-space n . (x - p - u t) >= 0
      double d[3], vr[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        d[c] = m.X[c * m.CN + j] - fma(P.wall_u[k][c], t, P.wall_p[k][c]);
        vr[c] = m.VN[c * m.CN + j] - P.wall_u[k][c];
      }
      const double* nn = P.wall_n[k];
      const double delta = rc->radius - fma(d[0], nn[0], fma(d[1], nn[1], d[2] * nn[2]));
      if (!(delta > 0.0)) continue;
      const double vn = fma(vr[0], nn[0], fma(vr[1], nn[1], vr[2] * nn[2]));
      double fn = P.wall_k * delta - P.wall_c * vn;
      if (fn < 0.0) fn = 0.0;
      double vt[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) vt[c] = vr[c] - vn * nn[c];
      const double sp = sqrt(fma(vt[0], vt[0], fma(vt[1], vt[1], vt[2] * vt[2])));
      const double fr = (P.wall_mu > 0.0 && fn > 0.0) ? -P.wall_mu * fn / fmax(sp, P.wall_vslip) : 0.0;
#pragma unroll
      for (int c = 0; c < 3; ++c) F[c] += fn * nn[c] + fr * vt[c];
    }
    if (MODE == MODE_RHS) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double vj = m.VN[c * m.CN + j];
        double a = fma(F[c], im, -dl * vj);
        if (P.has_gravity) a += P.gravity[c];
        acc_v[c * P.N + gn] = held ? 0.0 : a;
      }
    } else {
      // v += dt (F/m - c v + g)  as  v (1 - dt c) + (dt/m) F + dt g  (keep = 1 without damping)
      const double dtim = dt * im;
      if (FS & kFeatDamp) {
        const double keep = P.has_damp_lin ? fma(-dt, dl, 1.0) : 1.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const double vj = m.VN[c * m.CN + j];
          const double base = P.has_damp_lin ? (P.has_gravity ? fma(vj, keep, dtg[c]) : vj * keep)
                                             : (P.has_gravity ? fma(dt, P.gravity[c], vj) : vj);
          m.VN[c * m.CN + j] = held ? 0.0 : fma(F[c], dtim, base);
        }
      } else {
        // no damping: v + dt g as one FMA, as the general kernel forms it (gravity zero: v)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          m.VN[c * m.CN + j] = held ? 0.0 : fma(F[c], dtim, fma(dt, P.gravity[c], m.VN[c * m.CN + j]));
      }
      // the following kinematic half/full step of this node (it reads only its own x, v)
      if (h != 0.0) kin_node(P, pk, m, j, h);
    }
  }
}

// Time-dependent values of a step at its force time t, shared by the whole block: the base
// couple of every rod, the magnetic field and t itself.  Written by the last threads of the
// block (idle in the element loops of small packs), without a barrier: the caller orders them
// before their readers.
__device__ __forceinline__ bool has_time_values(const StepParams& P) {
  return P.has_act || P.magnet != nullptr || P.arc0 != nullptr || P.n_walls > 0;
}

__device__ __forceinline__ void time_values(const StepParams& P, const Pack& pk, Smem& m, double t) {
  const int rev = m.ts - 1 - m.t0;
  if (P.has_act) {
    for (int r = rev; r < pk.nrods; r += m.ts) {
      const RodConst* rc = P.rods + m.grod[r];
      const double amp = rc->act_amp;
      m.ACT[r] = (amp != 0.0) ? amp * sin(fma(rc->act_omega, t, rc->act_phase)) : 0.0;
    }
  }
  if (rev == 0 && (P.magnet != nullptr || P.arc0 != nullptr || P.n_walls > 0)) {
    if (P.magnet) {
      const double co = cos(P.field_omega * t), si = sin(P.field_omega * t);
#pragma unroll
      for (int c = 0; c < 3; ++c) m.BF[c] = P.field_b0[c] + P.field_bc[c] * co + P.field_bs[c] * si;
    }
    m.BF[3] = t;
  }
}

// The same, followed by a barrier (other warps read them in the next stage).
__device__ __forceinline__ void actuation_values(const StepParams& P, const Pack& pk, Smem& m, double t) {
  if (!has_time_values(P)) return;
  time_values(P, pk, m, t);
  stage_sync(m);
}

// Copy a pack's state and constants into shared memory and build the item -> rod maps.
__device__ __forceinline__ void stage_pack(const StepParams& P, const Pack& pk, Smem& m) {
  const int Ep = pk.nelem, Np = pk.nnode, Rp = pk.nrods, Vp = pk.nvor;
  for (int r = m.t0; r < Rp; r += m.ts) {
    int g, rel;
    if (pk.listed) {
      const int2 e = P.pack_rods[pk.list_off + r];
      g = e.x;
      rel = e.y;
    } else {
      g = pk.rod0 + r;
      rel = P.rods[g].elem0 - pk.elem0;
    }
    const RodConst& rc = P.rods[g];
    m.rel0[r] = rel;
    m.grod[r] = g;
    m.dE[r] = rc.elem0 - rel;
    m.dN[r] = rc.node0 - rel - r;
    m.dV[r] = rc.elem0 - g - rel + r;
  }
  if (m.t0 == 0) m.rel0[Rp] = Ep;
  stage_sync(m);
  for (int i = m.t0; i < Ep; i += m.ts) {
    const int r = find_rod(m.rel0, Rp, i);
    const int ge = i + m.dE[r];
    m.erod[i] = (short)r;
#pragma unroll
    for (int a = 0; a < 9; ++a) m.QQ[a * m.CE + i] = P.Q[a * P.E + ge];
#pragma unroll
    for (int c = 0; c < 3; ++c) m.WW[c * m.CE + i] = P.w[c * P.E + ge];
  }
  for (int j = m.t0; j < Np; j += m.ts) {
    // node j belongs to rod r with rel0[r] + r <= j
    int lo = 0, hi = Rp - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (m.rel0[mid] + mid <= j) lo = mid; else hi = mid - 1;
    }
    m.nrod[j] = (short)lo;
    const int gn = j + m.dN[lo];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m.X[c * m.CN + j] = P.x[c * P.N + gn];
      m.VN[c * m.CN + j] = P.v[c * P.N + gn];
    }
  }
  for (int k = m.t0; k < Vp; k += m.ts) {
    int lo = 0, hi = Rp - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (m.rel0[mid] - mid <= k) lo = mid; else hi = mid - 1;
    }
    m.vrod[k] = (short)lo;
  }
  stage_sync(m);

}

}  // namespace
}  // namespace rod
