// rod_adjoint.cu -- hand-written adjoint (reverse mode) of one FP64 rod step, sm_103a.
//
// Given the state at the start of a step and the adjoint of the state at its end, a thread
// block re-runs the forward step of its pack with the forward kernel's own stages (same
// arithmetic, shared memory), then walks the stages backwards:
//   second kinematic half   Q' = exp(-h[w']x) Qh, x' = xh + h v'
//   rate update             v' = v + dt a, w' = w + dt alpha (clamped items fixed)
//   right-hand side         a = F/m, alpha = e J^{-1} tau (Eq. 1a, 1b) through the internal
//                           force, shear/bend/twist couples, transport couples, damping
//   first kinematic half    Qh = exp(-h[w]x) Q, xh = x + h v
// producing the adjoint of the start state and accumulating the gradients with respect to
// the rest curvature kappa0 (enters m = B(kappa - kappa0)) and the element couples C (enter
// tau).  Neighbour contributions (difference and averaging operators) are exchanged through
// shared memory exactly like the forward stages.  The exponential and logarithm derivatives
// use the derivatives of the same Taylor series (or of sin/cos/atan2 for large angles).
// The directors' adjoint is taken with respect to their nine entries.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "rod_adjoint.h"
#include "rod_step_device.cuh"

namespace rod {
namespace {

// d a / d(th^2) and d b / d(th^2) of a = sin th / th, b = (1 - cos th) / th^2: the derivatives
// of the series that rot_coeffs evaluates, cut by the same warp-uniform rule (two terms below
// th^2 = 2^-20, four below 2^-10), otherwise of the full series or of sin and cos.
__device__ __forceinline__ void rot_coeff_derivs(double th2, double& da, double& db) {
  const unsigned mx = __reduce_max_sync(__activemask(), hi_word(th2));
  if (mx < kHi2m20) {
    da = -1.0 / 6.0;
    db = -1.0 / 24.0;
  } else if (mx < kHi2m10) {
    da = fma(fma(th2, 3.0 * (-1.0 / 5040.0), 2.0 / 120.0), th2, -1.0 / 6.0);
    db = fma(fma(th2, 3.0 * (-1.0 / 40320.0), 2.0 / 720.0), th2, -1.0 / 24.0);
  } else if (th2 <= 0.25) {
    // term n of a: (-1)^n th^(2n) / (2n+1)!, derivative n (-1)^n th^(2n-2) / (2n+1)!
    da = 7.0 * (-1.0 / 1307674368000.0);
    da = fma(da, th2, 6.0 / 6227020800.0);
    da = fma(da, th2, 5.0 * (-1.0 / 39916800.0));
    da = fma(da, th2, 4.0 / 362880.0);
    da = fma(da, th2, 3.0 * (-1.0 / 5040.0));
    da = fma(da, th2, 2.0 / 120.0);
    da = fma(da, th2, -1.0 / 6.0);
    db = 7.0 * (-1.0 / 20922789888000.0);
    db = fma(db, th2, 6.0 / 87178291200.0);
    db = fma(db, th2, 5.0 * (-1.0 / 479001600.0));
    db = fma(db, th2, 4.0 / 3628800.0);
    db = fma(db, th2, 3.0 * (-1.0 / 40320.0));
    db = fma(db, th2, 2.0 / 720.0);
    db = fma(db, th2, -1.0 / 24.0);
  } else {
    const double th = sqrt(th2);
    double s, c;
    sincos(th, &s, &c);
    da = (th * c - s) / (2.0 * th2 * th);
    db = (th * s - 2.0 * (1.0 - c)) / (2.0 * th2 * th2);
  }
}

// d f / d(s^2) of f = asin(s)/s (13-term series, as the forward).
__device__ __forceinline__ double dasin_over_s(double s2) {
  double f = 12.0 * (676039.0 / 104857600.0);
  f = fma(f, s2, 11.0 * (88179.0 / 12058624.0));
  f = fma(f, s2, 10.0 * (46189.0 / 5505024.0));
  f = fma(f, s2, 9.0 * (12155.0 / 1245184.0));
  f = fma(f, s2, 8.0 * (6435.0 / 557056.0));
  f = fma(f, s2, 7.0 * (143.0 / 10240.0));
  f = fma(f, s2, 6.0 * (231.0 / 13312.0));
  f = fma(f, s2, 5.0 * (63.0 / 2816.0));
  f = fma(f, s2, 4.0 * (35.0 / 1152.0));
  f = fma(f, s2, 3.0 * (5.0 / 112.0));
  f = fma(f, s2, 2.0 * (3.0 / 40.0));
  f = fma(f, s2, 1.0 / 6.0);
  return f;
}

// R = exp([phi]x) entries (row-major) and its coefficients.
struct Rot {
  double R[9];
  double a, b, th2;
};

__device__ __forceinline__ Rot make_rot(const double p[3]) {
  Rot r;
  r.th2 = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
  rot_coeffs(r.th2, r.a, r.b);   // the forward's series, cut per warp
  const double c0 = 1.0 - r.b * r.th2;
  r.R[0] = c0 + r.b * p[0] * p[0];
  r.R[4] = c0 + r.b * p[1] * p[1];
  r.R[8] = c0 + r.b * p[2] * p[2];
  r.R[1] = r.b * p[0] * p[1] - r.a * p[2];
  r.R[3] = r.b * p[1] * p[0] + r.a * p[2];
  r.R[2] = r.b * p[0] * p[2] + r.a * p[1];
  r.R[6] = r.b * p[2] * p[0] - r.a * p[1];
  r.R[5] = r.b * p[1] * p[2] - r.a * p[0];
  r.R[7] = r.b * p[2] * p[1] + r.a * p[0];
  return r;
}

// Adjoint of Y = R(phi) X for the 3x3 matrices X (input) and Y (output): Xbar = R^T Ybar and the
// gradient with respect to phi, from d(R q)/d phi_k for each column q of X:
//   phibar = 2 phi [ -(b' th^2 + b) S1 + a' S2 + b' S3 ] + a V1 + b (V2 + V3)
//   S1 = sum_c ybar_c . q_c,  S2 = sum_c ybar_c . (phi x q_c),  S3 = sum_c (phi . q_c)(ybar_c . phi)
//   V1 = sum_c q_c x ybar_c,  V2 = sum_c (phi . q_c) ybar_c,   V3 = sum_c (ybar_c . phi) q_c
__device__ __forceinline__ void rot_adjoint(const double p[3], const Rot& r, const double X[9], const double Yb[9],
                                            double Xb[9], double pb[3]) {
  double da, db;
  rot_coeff_derivs(r.th2, da, db);
  double S1 = 0, S2 = 0, S3 = 0, V1[3] = {0, 0, 0}, V2[3] = {0, 0, 0}, V3[3] = {0, 0, 0};
  for (int c = 0; c < 3; ++c) {
    const double q[3] = {X[c], X[3 + c], X[6 + c]};
    const double y[3] = {Yb[c], Yb[3 + c], Yb[6 + c]};
    const double pxq[3] = {p[1] * q[2] - p[2] * q[1], p[2] * q[0] - p[0] * q[2], p[0] * q[1] - p[1] * q[0]};
    const double pq = p[0] * q[0] + p[1] * q[1] + p[2] * q[2];
    const double yp = y[0] * p[0] + y[1] * p[1] + y[2] * p[2];
    S1 += y[0] * q[0] + y[1] * q[1] + y[2] * q[2];
    S2 += y[0] * pxq[0] + y[1] * pxq[1] + y[2] * pxq[2];
    S3 += pq * yp;
    V1[0] += q[1] * y[2] - q[2] * y[1];
    V1[1] += q[2] * y[0] - q[0] * y[2];
    V1[2] += q[0] * y[1] - q[1] * y[0];
    for (int k = 0; k < 3; ++k) {
      V2[k] += pq * y[k];
      V3[k] += yp * q[k];
    }
    // Xbar column c = R^T ybar_c
    for (int k = 0; k < 3; ++k) Xb[3 * k + c] = r.R[k] * y[0] + r.R[3 + k] * y[1] + r.R[6 + k] * y[2];
  }
  const double sc = 2.0 * (-(db * r.th2 + r.b) * S1 + da * S2 + db * S3);
  for (int k = 0; k < 3; ++k) pb[k] = sc * p[k] + r.a * V1[k] + r.b * (V2[k] + V3[k]);
}

struct AdjSmem {
  double *Q0, *QH, *W0, *V0;         // forward values kept for the reverse sweep
  double *XB, *VB, *FB;              // node adjoints: xh (then x), v, F
  double *QB, *WB, *TAUB, *DVB;      // element adjoints: Qh (then Q), w, tau, dv
  double *LB, *LBL, *LV, *RS;        // element: lbar (3), ellbar, l (3), 1/ell
  double *VQA, *VQB, *EPSB;          // Voronoi: contributions to Qh of elements k and k+1, ell
};

__device__ __forceinline__ AdjSmem carve_adj(double* base, const Smem& m) {
  AdjSmem a;
  double* p = base;
  a.Q0 = p; p += 9 * m.CE;
  a.QH = p; p += 9 * m.CE;
  a.W0 = p; p += 3 * m.CE;
  a.V0 = p; p += 3 * m.CN;
  a.XB = p; p += 3 * m.CN;
  a.VB = p; p += 3 * m.CN;
  a.FB = p; p += 3 * m.CN;
  a.QB = p; p += 9 * m.CE;
  a.WB = p; p += 3 * m.CE;
  a.TAUB = p; p += 3 * m.CE;
  a.DVB = p; p += 3 * m.CE;
  a.LB = p; p += 3 * m.CE;
  a.LBL = p; p += m.CE;
  a.LV = p; p += 3 * m.CE;
  a.RS = p; p += m.CE;
  a.VQA = p; p += 9 * m.CV;
  a.VQB = p; p += 9 * m.CV;
  a.EPSB = p; p += m.CV;
  return a;
}

__global__ void __launch_bounds__(256) adjoint_kernel(AdjointParams A, LaunchShape S) {
  extern __shared__ double smem_d[];
  const StepParams& P = A.P;
  const Pack pk = P.packs[blockIdx.x];
  Smem m = carve(smem_d, S);
  AdjSmem a = carve_adj(smem_d + A.fwd_smem_doubles, m);
  const int Ep = pk.nelem, Np = pk.nnode, Vp = pk.nvor;
  const double dt = A.dt, h = 0.5 * A.dt;

  // ---- forward state at the step start, adjoint of the step end
  stage_pack(P, pk, m);
  for (int i = threadIdx.x; i < Ep; i += blockDim.x) {
    const int ge = pk.elem0 + i;
    for (int k = 0; k < 9; ++k) {
      a.Q0[k * m.CE + i] = m.QQ[k * m.CE + i];
      a.QB[k * m.CE + i] = A.aQ[k * P.E + ge];
    }
    for (int c = 0; c < 3; ++c) {
      a.W0[c * m.CE + i] = m.WW[c * m.CE + i];
      a.WB[c * m.CE + i] = A.aw[c * P.E + ge];
    }
  }
  for (int j = threadIdx.x; j < Np; j += blockDim.x) {
    const int gn = pk.node0 + j;
    for (int c = 0; c < 3; ++c) {
      a.V0[c * m.CN + j] = m.VN[c * m.CN + j];
      a.XB[c * m.CN + j] = A.ax[c * P.N + gn];
      a.VB[c * m.CN + j] = A.av[c * P.N + gn];
    }
  }
  __syncthreads();

  // ---- forward recompute of the step (first half, right-hand side, rate update)
  kinematic(P, pk, m, h);
  __syncthreads();
  for (int i = threadIdx.x; i < Ep; i += blockDim.x)
    for (int k = 0; k < 9; ++k) a.QH[k * m.CE + i] = m.QQ[k * m.CE + i];
  actuation_values(P, pk, m, A.t + h);
  stage_elements(P, pk, m);
  __syncthreads();
  stage_voronoi(P, pk, m);
  __syncthreads();
  stage_rotation<MODE_STEPS>(P, pk, m, dt, 0.0, nullptr);   // WW <- w'
  stage_translation<MODE_STEPS>(P, pk, m, dt, nullptr, A.t + h);   // VN <- v'
  __syncthreads();

  // ---- reverse of the second kinematic half (h): Q' = R(-h w') Qh, x' = xh + h v'
  for (int i = threadIdx.x; i < Ep; i += blockDim.x) {
    const int r = m.erod[i];
    const bool held = (i == m.rel0[r]) && P.rods[pk.rod0 + r].clamp;
    double Yb[9], Xb[9], X[9], pb[3];
    for (int k = 0; k < 9; ++k) {
      Yb[k] = a.QB[k * m.CE + i];
      X[k] = a.QH[k * m.CE + i];
    }
    if (held) {
      for (int k = 0; k < 9; ++k) a.QB[k * m.CE + i] = 0.0;
      continue;
    }
    const double p[3] = {-h * m.WW[i], -h * m.WW[m.CE + i], -h * m.WW[2 * m.CE + i]};
    const Rot rt = make_rot(p);
    rot_adjoint(p, rt, X, Yb, Xb, pb);
    for (int k = 0; k < 9; ++k) a.QB[k * m.CE + i] = Xb[k];
    for (int c = 0; c < 3; ++c) a.WB[c * m.CE + i] += -h * pb[c];
  }
  for (int j = threadIdx.x; j < Np; j += blockDim.x) {
    const int r = m.nrod[j];
    const bool held = (j == m.rel0[r] + r) && P.rods[pk.rod0 + r].clamp;
    for (int c = 0; c < 3; ++c) {
      const double xb = held ? 0.0 : a.XB[c * m.CN + j];
      a.XB[c * m.CN + j] = xb;                      // now: adjoint of xh
      a.VB[c * m.CN + j] += h * xb;                 // now: adjoint of v'
    }
  }
  __syncthreads();

  // ---- reverse of the rate update and of alpha = e J^{-1} tau, a = F/m - c v + g
  for (int i = threadIdx.x; i < Ep; i += blockDim.x) {
    const int r = m.erod[i];
    const int g = pk.rod0 + r;
    const RodConst* rc = P.rods + g;
    const int first = m.rel0[r];
    const int nr = m.rel0[r + 1] - first;
    const int li = i - first, k = i - r;
    const bool held = (li == 0) && rc->clamp;
    const bool hasR = li < nr - 1, hasL = li > 0;
    double tau[3];
    element_couple<kFeatAll>(P, m, i, k, hasR, hasL, tau);
    double ebar = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double wb = held ? 0.0 : a.WB[c * m.CE + i];
      const double alpha_b = dt * wb;
      const double jinv = P.inv_rl[pk.elem0 + i] * rc->inv_rhoI[c];
      const double taub = m.EDIL[i] * rc->inv_rhoI[c] * alpha_b;   // EDIL = e / rl
      ebar += jinv * tau[c] * alpha_b;
      a.TAUB[c * m.CE + i] = taub;
      a.WB[c * m.CE + i] = wb;                       // now: adjoint of w (through w' = w + dt alpha)
      A.g_couple[c * P.E + pk.elem0 + i] += taub;    // tau contains C directly
    }
    a.LBL[i] = ebar * P.inv_rl[pk.elem0 + i];                      // e = ell / rl
  }
  for (int j = threadIdx.x; j < Np; j += blockDim.x) {
    const int r = m.nrod[j];
    const RodConst* rc = P.rods + pk.rod0 + r;
    const bool held = (j == m.rel0[r] + r) && rc->clamp;
    for (int c = 0; c < 3; ++c) {
      const double vb = held ? 0.0 : a.VB[c * m.CN + j];
      const double abar = dt * vb;
      a.FB[c * m.CN + j] = abar * P.inv_m[pk.node0 + j];
      a.VB[c * m.CN + j] = vb - rc->damp_lin * abar;   // adjoint of v (rate update + damping)
    }
    // walls: F = fn n + fr vt with fn = k delta - c (v - u).n, delta = r - n.(xh - p - u t),
    // vt the tangential part of v - u, fr = -mu fn / max(|vt|, v_slip) (active contacts only)
    for (int kw = 0; kw < P.n_walls && !held; ++kw) {
      const double tw = A.t + h;
      const double* nn = P.wall_n[kw];
      double d[3], vr[3], Fb[3];
      for (int c = 0; c < 3; ++c) {
        d[c] = m.X[c * m.CN + j] - fma(P.wall_u[kw][c], tw, P.wall_p[kw][c]);
        vr[c] = a.V0[c * m.CN + j] - P.wall_u[kw][c];
        Fb[c] = a.FB[c * m.CN + j];
      }
      const double delta = rc->radius - fma(d[0], nn[0], fma(d[1], nn[1], d[2] * nn[2]));
      if (!(delta > 0.0)) continue;
      const double vn = fma(vr[0], nn[0], fma(vr[1], nn[1], vr[2] * nn[2]));
      const double fn = P.wall_k * delta - P.wall_c * vn;
      if (!(fn > 0.0)) continue;
      double vt[3];
      for (int c = 0; c < 3; ++c) vt[c] = vr[c] - vn * nn[c];
      const double sp = sqrt(fma(vt[0], vt[0], fma(vt[1], vt[1], vt[2] * vt[2])));
      const double s_n = Fb[0] * nn[0] + Fb[1] * nn[1] + Fb[2] * nn[2];
      double fnb = s_n, vtb[3] = {0.0, 0.0, 0.0};
      if (P.wall_mu > 0.0) {
        const double den = fmax(sp, P.wall_vslip);
        const double fr = -P.wall_mu * fn / den;
        const double g = Fb[0] * vt[0] + Fb[1] * vt[1] + Fb[2] * vt[2];
        fnb += -P.wall_mu / den * g;
        for (int c = 0; c < 3; ++c) vtb[c] = fr * Fb[c];
        if (sp > P.wall_vslip) {
          const double spb = P.wall_mu * fn / (den * den) * g;
          for (int c = 0; c < 3; ++c) vtb[c] += spb * vt[c] / sp;
        }
      }
      // vt = vr - vn n;  fn = k delta - c vn;  vn = vr . n;  delta = r - n . d
      const double ntb = nn[0] * vtb[0] + nn[1] * vtb[1] + nn[2] * vtb[2];
      const double vnb = -ntb - P.wall_c * fnb;
      const double deltab = P.wall_k * fnb;
      for (int c = 0; c < 3; ++c) {
        a.VB[c * m.CN + j] += vtb[c] + vnb * nn[c];
        a.XB[c * m.CN + j] += -deltab * nn[c];
      }
    }
  }
  __syncthreads();

  // ---- reverse of the element terms: internal force, shear couple, transport, damping
  for (int i = threadIdx.x; i < Ep; i += blockDim.x) {
    const int r = m.erod[i];
    const RodConst* rc = P.rods + pk.rod0 + r;
    const int j = i + r;
    const int ge = pk.elem0 + i;
    double l[3], dv[3], q[9], w[3], taub[3];
    for (int c = 0; c < 3; ++c) {
      l[c] = m.X[c * m.CN + j + 1] - m.X[c * m.CN + j];
      dv[c] = a.V0[c * m.CN + j + 1] - a.V0[c * m.CN + j];
      w[c] = a.W0[c * m.CE + i];
      taub[c] = a.TAUB[c * m.CE + i];
    }
    for (int k = 0; k < 9; ++k) q[k] = a.QH[k * m.CE + i];
    const double ll = l[0] * l[0] + l[1] * l[1] + l[2] * l[2];
    const double rs = rsqrt(ll);
    const double irl = P.inv_rl[pk.elem0 + i];
    const double rl = P.rest_len[ge];
    const double ie = rl * rs;
    double Ql[3], sg[3], n[3];
    for (int b = 0; b < 3; ++b) Ql[b] = q[3 * b] * l[0] + q[3 * b + 1] * l[1] + q[3 * b + 2] * l[2];
    sg[0] = Ql[0] * irl;
    sg[1] = Ql[1] * irl;
    sg[2] = Ql[2] * irl - 1.0;
    if (P.rest_sigma)
      for (int c = 0; c < 3; ++c) sg[c] -= P.rest_sigma[c * P.E + ge];
    for (int c = 0; c < 3; ++c) n[c] = (rc->S[c] * ie) * sg[c];
    const double ldv = l[0] * dv[0] + l[1] * dv[1] + l[2] * dv[2];
    const double edot = ldv * rs * irl;
    double Jw[3], Jwe[3];
    for (int c = 0; c < 3; ++c) {
      Jw[c] = rc->rhoI[c] * rl * w[c];
      Jwe[c] = Jw[c] * ie;
    }
    const double k2 = ie * ie * edot;
    // N-bar = F-bar(node i) - F-bar(node i+1)
    double Nb[3];
    for (int c = 0; c < 3; ++c) Nb[c] = a.FB[c * m.CN + j] - a.FB[c * m.CN + j + 1];
    // tau = (Ql x n) + (Jwe x w) + Jw (k2 - c_rot) + C
    double Jwb[3], Jweb[3], wb[3] = {0, 0, 0}, nb[3], Qlb[3];
    Jweb[0] = w[1] * taub[2] - w[2] * taub[1];
    Jweb[1] = w[2] * taub[0] - w[0] * taub[2];
    Jweb[2] = w[0] * taub[1] - w[1] * taub[0];
    wb[0] += taub[1] * Jwe[2] - taub[2] * Jwe[1];
    wb[1] += taub[2] * Jwe[0] - taub[0] * Jwe[2];
    wb[2] += taub[0] * Jwe[1] - taub[1] * Jwe[0];
    const double k2b = Jw[0] * taub[0] + Jw[1] * taub[1] + Jw[2] * taub[2];
    for (int c = 0; c < 3; ++c) Jwb[c] = (k2 - rc->damp_rot) * taub[c] + ie * Jweb[c];
    double ieb = (Jw[0] * Jweb[0] + Jw[1] * Jweb[1] + Jw[2] * Jweb[2]) + 2.0 * ie * edot * k2b;
    const double edotb = ie * ie * k2b;
    Qlb[0] = n[1] * taub[2] - n[2] * taub[1];
    Qlb[1] = n[2] * taub[0] - n[0] * taub[2];
    Qlb[2] = n[0] * taub[1] - n[1] * taub[0];
    nb[0] = taub[1] * Ql[2] - taub[2] * Ql[1];
    nb[1] = taub[2] * Ql[0] - taub[0] * Ql[2];
    nb[2] = taub[0] * Ql[1] - taub[1] * Ql[0];
    // N = Qh^T n
    double Qhb[9];
    for (int aa = 0; aa < 3; ++aa) {
      nb[aa] += q[3 * aa] * Nb[0] + q[3 * aa + 1] * Nb[1] + q[3 * aa + 2] * Nb[2];
      for (int b = 0; b < 3; ++b) Qhb[3 * aa + b] = n[aa] * Nb[b];
    }
    if (P.magnet) {
      // magnetic couple rl (m x (Qh b)): d/dQh_ab of taub . (m x Qh b) = (taub x m)_a b_b rl
      double mg[3], lxm[3];
      for (int c = 0; c < 3; ++c) mg[c] = rl * P.magnet[c * P.E + ge];
      lxm[0] = taub[1] * mg[2] - taub[2] * mg[1];
      lxm[1] = taub[2] * mg[0] - taub[0] * mg[2];
      lxm[2] = taub[0] * mg[1] - taub[1] * mg[0];
      for (int aa = 0; aa < 3; ++aa)
        for (int b = 0; b < 3; ++b) Qhb[3 * aa + b] += lxm[aa] * m.BF[b];
    }
    // n = (S ie) sigma, sigma = Ql / rl - e3 - sigma0
    for (int c = 0; c < 3; ++c) {
      const double sgb = rc->S[c] * ie * nb[c];
      ieb += rc->S[c] * sg[c] * nb[c];
      Qlb[c] += irl * sgb;
    }
    // Ql = Qh l
    double lb[3] = {0, 0, 0};
    for (int aa = 0; aa < 3; ++aa)
      for (int b = 0; b < 3; ++b) {
        Qhb[3 * aa + b] += Qlb[aa] * l[b];
        lb[b] += q[3 * aa + b] * Qlb[aa];
      }
    // edot = (l . dv) rs / rl
    const double ce = rs * irl * edotb;
    double rsb = ldv * irl * edotb + rl * ieb;      // ie = rl rs
    for (int c = 0; c < 3; ++c) {
      lb[c] += ce * dv[c];
      a.DVB[c * m.CE + i] = ce * l[c];
    }
    // Jw = rho I rl w
    for (int c = 0; c < 3; ++c) wb[c] += rc->rhoI[c] * rl * Jwb[c];
    // rs = 1/ell: ellbar -= rs^2 rsbar
    a.LBL[i] += -rs * rs * rsb;
    for (int k = 0; k < 9; ++k) a.QB[k * m.CE + i] += Qhb[k];
    for (int c = 0; c < 3; ++c) {
      a.WB[c * m.CE + i] += wb[c];
      a.LB[c * m.CE + i] = lb[c];
      a.LV[c * m.CE + i] = l[c];
    }
    a.RS[i] = rs;
  }
  __syncthreads();

  // ---- reverse of the Voronoi terms: curvature (rotation logarithm), bend/twist couple
  for (int k = threadIdx.x; k < Vp; k += blockDim.x) {
    const int r = m.vrod[k];
    const RodConst* rc = P.rods + pk.rod0 + r;
    const int i = k + r;
    const int gv = pk.vor0 + k;
    double qa[9], qb[9];
    for (int t = 0; t < 9; ++t) {
      qa[t] = a.QH[t * m.CE + i];
      qb[t] = a.QH[t * m.CE + i + 1];
    }
    double u[3];
    u[0] = (qb[6] * qa[3] + qb[7] * qa[4] + qb[8] * qa[5]) - (qb[3] * qa[6] + qb[4] * qa[7] + qb[5] * qa[8]);
    u[1] = (qb[0] * qa[6] + qb[1] * qa[7] + qb[2] * qa[8]) - (qb[6] * qa[0] + qb[7] * qa[1] + qb[8] * qa[2]);
    u[2] = (qb[3] * qa[0] + qb[4] * qa[1] + qb[5] * qa[2]) - (qb[0] * qa[3] + qb[1] * qa[4] + qb[2] * qa[5]);
    double tr = 0.0;
    for (int t = 0; t < 9; ++t) tr += qb[t] * qa[t];
    const double s2 = 0.25 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    const double cth = 0.5 * (tr - 1.0);
    double f, dfds2, dfdc = 0.0;
    // theta / sin theta and its derivative: the asin(s)/s series cut per warp like the forward's
    // (three terms below s^2 = 2^-20, six below 2^-10, when every lane's angle is below 90 deg)
    const unsigned act = __activemask();
    const bool series = __all_sync(act, s2 <= 0.0625 && cth > 0.0);
    const unsigned mx = __reduce_max_sync(act, hi_word(s2));
    if (series && mx < kHi2m20) {
      f = fma(fma(s2, 3.0 / 40.0, 1.0 / 6.0), s2, 1.0);
      dfds2 = fma(s2, 2.0 * (3.0 / 40.0), 1.0 / 6.0);
    } else if (series && mx < kHi2m10) {
      f = fma(fma(fma(fma(fma(s2, 63.0 / 2816.0, 35.0 / 1152.0), s2, 5.0 / 112.0), s2, 3.0 / 40.0), s2, 1.0 / 6.0), s2, 1.0);
      dfds2 = fma(fma(fma(fma(s2, 5.0 * (63.0 / 2816.0), 4.0 * (35.0 / 1152.0)), s2, 3.0 * (5.0 / 112.0)), s2,
                      2.0 * (3.0 / 40.0)), s2, 1.0 / 6.0);
    } else if (s2 <= 0.0625 && cth > 0.0) {
      f = asin_over_s(s2);
      dfds2 = dasin_over_s(s2);
    } else {
      const double sn = sqrt(s2);
      const double th = atan2(sn, cth);
      const double den = s2 + cth * cth;
      if (sn > 0.0) {
        f = th / sn;
        dfds2 = (cth / den * sn - th) / (s2 * 2.0 * sn);  // (d theta/ds s - theta)/s^2 / (2 s)
        dfdc = -1.0 / den;
      } else {
        f = 1.0;
        dfds2 = 0.0;
      }
    }
    const double i2D = P.inv_2D[gv];
    const double Dh = P.Dhat[gv];
    const double kf = -f * i2D;
    double kap[3] = {kf * u[0], kf * u[1], kf * u[2]};
    const double eps = (m.ELL[i] + m.ELL[i + 1]) * i2D;
    const double ieps = rcp_nr(eps);
    const double ie3 = ieps * ieps * ieps;
    double mk[3];
    for (int c = 0; c < 3; ++c)
      mk[c] = rc->B[c] * (kap[c] - (P.rest_kappa ? P.rest_kappa[c * P.V + gv] : 0.0));
    const double y[3] = {kap[1] * mk[2] - kap[2] * mk[1], kap[2] * mk[0] - kap[0] * mk[2],
                         kap[0] * mk[1] - kap[1] * mk[0]};
    // P-bar = tau-bar_i - tau-bar_{i+1}, T-bar = (tau-bar_i + tau-bar_{i+1}) / 2
    double Pb[3], Tb[3];
    for (int c = 0; c < 3; ++c) {
      const double t0 = a.TAUB[c * m.CE + i], t1 = a.TAUB[c * m.CE + i + 1];
      Pb[c] = t0 - t1;
      Tb[c] = 0.5 * (t0 + t1);
    }
    double mkb[3], kapb[3], yb[3];
    double ie3b = 0.0;
    for (int c = 0; c < 3; ++c) {
      mkb[c] = ie3 * Pb[c];
      ie3b += mk[c] * Pb[c] + Dh * y[c] * Tb[c];
      yb[c] = Dh * ie3 * Tb[c];
    }
    // y = kap x mk
    kapb[0] = mk[1] * yb[2] - mk[2] * yb[1];
    kapb[1] = mk[2] * yb[0] - mk[0] * yb[2];
    kapb[2] = mk[0] * yb[1] - mk[1] * yb[0];
    mkb[0] += yb[1] * kap[2] - yb[2] * kap[1];
    mkb[1] += yb[2] * kap[0] - yb[0] * kap[2];
    mkb[2] += yb[0] * kap[1] - yb[1] * kap[0];
    for (int c = 0; c < 3; ++c) {
      kapb[c] += rc->B[c] * mkb[c];
      A.g_kappa0[c * P.V + gv] += -rc->B[c] * mkb[c];
    }
    // eps = (ell_i + ell_{i+1}) / (2D), ie3 = eps^-3
    const double epsb = -3.0 * ie3 * ieps * ie3b;
    a.EPSB[k] = epsb * i2D;
    // kappa = -f(s^2, c) u / (2D), s^2 = |u|^2 / 4, c = (tr - 1) / 2
    const double uk = u[0] * kapb[0] + u[1] * kapb[1] + u[2] * kapb[2];
    double ub[3];
    for (int c = 0; c < 3; ++c) ub[c] = kf * kapb[c] - i2D * dfds2 * uk * 0.5 * u[c];
    const double trb = -i2D * dfdc * uk * 0.5;
    // u0 = d3'.d2 - d2'.d3, u1 = d1'.d3 - d3'.d1, u2 = d2'.d1 - d1'.d2 (' = element i+1)
    double gA[9], gB[9];
    for (int c = 0; c < 3; ++c) {
      const double a1 = qa[c], a2 = qa[3 + c], a3 = qa[6 + c];
      const double b1 = qb[c], b2 = qb[3 + c], b3 = qb[6 + c];
      gB[6 + c] = ub[0] * a2 - ub[1] * a1 + trb * a3;
      gB[3 + c] = -ub[0] * a3 + ub[2] * a1 + trb * a2;
      gB[c] = ub[1] * a3 - ub[2] * a2 + trb * a1;
      gA[3 + c] = ub[0] * b3 - ub[2] * b1 + trb * b2;
      gA[6 + c] = -ub[0] * b2 + ub[1] * b1 + trb * b3;
      gA[c] = -ub[1] * b3 + ub[2] * b2 + trb * b1;
    }
    for (int t = 0; t < 9; ++t) {
      a.VQA[t * m.CV + k] = gA[t];
      a.VQB[t * m.CV + k] = gB[t];
    }
  }
  __syncthreads();

  // ---- gather the Voronoi contributions into the elements, finish l-bar
  for (int i = threadIdx.x; i < Ep; i += blockDim.x) {
    const int r = m.erod[i];
    const int first = m.rel0[r];
    const int nr = m.rel0[r + 1] - first;
    const int li = i - first, k = i - r;
    const bool hasR = li < nr - 1, hasL = li > 0;
    double ellb = a.LBL[i] + (hasR ? a.EPSB[k] : 0.0) + (hasL ? a.EPSB[k - 1] : 0.0);
    const double rs = a.RS[i];
    for (int c = 0; c < 3; ++c) a.LB[c * m.CE + i] += ellb * rs * a.LV[c * m.CE + i];  // ell = |l|
    for (int t = 0; t < 9; ++t) {
      double add = 0.0;
      if (hasR) add += a.VQA[t * m.CV + k];
      if (hasL) add += a.VQB[t * m.CV + k - 1];
      a.QB[t * m.CE + i] += add;
    }
  }
  __syncthreads();

  // ---- nodes: l_i = xh_{i+1} - xh_i, dv_i = v_{i+1} - v_i; then the first kinematic half
  for (int j = threadIdx.x; j < Np; j += blockDim.x) {
    const int r = m.nrod[j];
    const int firstn = m.rel0[r] + r;
    const int nr = m.rel0[r + 1] - m.rel0[r];
    const int lj = j - firstn;
    const bool hasR = lj < nr, hasL = lj > 0;
    const int iR = j - r;
    const bool held = (lj == 0) && P.rods[pk.rod0 + r].clamp;
    for (int c = 0; c < 3; ++c) {
      double xb = a.XB[c * m.CN + j];
      double vb = a.VB[c * m.CN + j];
      if (hasR) {
        xb -= a.LB[c * m.CE + iR];
        vb -= a.DVB[c * m.CE + iR];
      }
      if (hasL) {
        xb += a.LB[c * m.CE + iR - 1];
        vb += a.DVB[c * m.CE + iR - 1];
      }
      // xh = x + h v (held node: xh fixed)
      const double xout = held ? 0.0 : xb;
      const double vout = held ? 0.0 : vb + h * xb;
      A.ax[c * P.N + pk.node0 + j] = xout;
      A.av[c * P.N + pk.node0 + j] = vout;
    }
  }
  for (int i = threadIdx.x; i < Ep; i += blockDim.x) {
    const int r = m.erod[i];
    const bool held = (i == m.rel0[r]) && P.rods[pk.rod0 + r].clamp;
    const int ge = pk.elem0 + i;
    if (held) {
      for (int t = 0; t < 9; ++t) A.aQ[t * P.E + ge] = 0.0;
      for (int c = 0; c < 3; ++c) A.aw[c * P.E + ge] = 0.0;
      continue;
    }
    double X[9], Yb[9], Xb[9], pb[3];
    for (int t = 0; t < 9; ++t) {
      X[t] = a.Q0[t * m.CE + i];
      Yb[t] = a.QB[t * m.CE + i];
    }
    const double p[3] = {-h * a.W0[i], -h * a.W0[m.CE + i], -h * a.W0[2 * m.CE + i]};
    const Rot rt = make_rot(p);
    rot_adjoint(p, rt, X, Yb, Xb, pb);
    for (int t = 0; t < 9; ++t) A.aQ[t * P.E + ge] = Xb[t];
    for (int c = 0; c < 3; ++c) A.aw[c * P.E + ge] = a.WB[c * m.CE + i] - h * pb[c];
  }
}

}  // namespace

size_t adjoint_smem_bytes(const LaunchShape& s) {
  const size_t CE = s.cap_elems, CR = s.cap_rods, CN = CE + CR, CV = CE;
  const size_t extra = 9 * CE + 9 * CE + 3 * CE + 3 * CN + 3 * CN + 3 * CN + 3 * CN + 9 * CE + 3 * CE + 3 * CE +
                       3 * CE + 3 * CE + CE + 3 * CE + CE + 9 * CV + 9 * CV + CV;
  return ((step_smem_bytes(s) + 7) / 8) * 8 + extra * sizeof(double);
}

cudaError_t launch_adjoint_kernel(const AdjointParams& A0, const LaunchShape& s, cudaStream_t st) {
  const size_t smem = adjoint_smem_bytes(s);
  cudaError_t e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  AdjointParams A = A0;
  A.fwd_smem_doubles = static_cast<int64_t>((step_smem_bytes(s) + 7) / 8);
  adjoint_kernel<<<A.P.n_packs, s.threads, smem, st>>>(A, s);
  return cudaGetLastError();
}

}  // namespace rod
