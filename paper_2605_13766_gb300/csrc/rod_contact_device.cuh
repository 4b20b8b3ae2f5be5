// rod_contact_device.cuh -- device functions of the rod-rod narrow phase shared by the contact
// kernels (rod_contact.cu) and the step kernel that evaluates the skin list's pairs itself
// (rod_step.cu).  Internal to librod.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "rod_contact.h"
#include "rod_internal.h"

namespace rod {
namespace {

// Largest number of segments one cell may hold; a denser cell (a collapsed or escaped
// configuration) latches ERR_OVERFLOW instead of running a quadratic search.
constexpr int kCellCap = 512;

// Closest points of P(s) = p0 + s d1, R(u) = q0 + u d2 on [0,1]^2 (minimise |r + s d1 - u d2|^2,
// r = p0 - q0): free minimiser s = (b f - c e)/(a e - b^2) clamped, u = (b s + f)/e; a clamped u
// re-solves s.  Parallel segments start from s = 0.  Quotients are taken as products with
// correctly rounded reciprocals (one per denominator): an FP64 division costs about three
// reciprocals on this part.
__device__ __forceinline__ void closest(const double* p0, const double* p1, const double* q0, const double* q1,
                                        double& s, double& u) {
  double d1[3], d2[3], r[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    d1[c] = p1[c] - p0[c];
    d2[c] = q1[c] - q0[c];
    r[c] = p0[c] - q0[c];
  }
  const double a = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2];
  const double e = d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2];
  const double f = d2[0] * r[0] + d2[1] * r[1] + d2[2] * r[2];
  if (a <= 0.0 && e <= 0.0) {
    s = 0.0;
    u = 0.0;
    return;
  }
  if (a <= 0.0) {
    s = 0.0;
    u = fmin(fmax(f * __drcp_rn(e), 0.0), 1.0);
    return;
  }
  const double c = d1[0] * r[0] + d1[1] * r[1] + d1[2] * r[2];
  if (e <= 0.0) {
    u = 0.0;
    s = fmin(fmax(-c * __drcp_rn(a), 0.0), 1.0);
    return;
  }
  const double b = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
  const double den = a * e - b * b;
  s = (den != 0.0) ? fmin(fmax((b * f - c * e) * __drcp_rn(den), 0.0), 1.0) : 0.0;
  u = (b * s + f) * __drcp_rn(e);
  if (u < 0.0) {
    u = 0.0;
    s = fmin(fmax(-c * __drcp_rn(a), 0.0), 1.0);
  } else if (u > 1.0) {
    u = 1.0;
    s = fmin(fmax((b - c) * __drcp_rn(a), 0.0), 1.0);
  }
}

struct PairForce {
  double fa[3], fb[3];
  bool hit;
};

// FP64 evaluation of one candidate pair (a, b) in canonical order (lower index first); returns
// the contributions to the two nodes of segment a.  Kept out of line: it runs only for the
// few candidates that survive the FP32 cull, and the scan loop stays small.
__device__ __noinline__ PairForce pair_force(const ContactArgs& A, int a, int ra, int b, int rb) {
  PairForce out;
  out.hit = false;
  const double rada = A.rods[ra].radius, radb = A.rods[rb].radius;
  const bool first = a < b;
  const int64_t na = a + ra, nb = b + rb;
  const int64_t nP = first ? na : nb, nQ = first ? nb : na;
  double P0[3], P1[3], Q0[3], Q1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    P0[c] = A.x[c * A.N + nP];
    P1[c] = A.x[c * A.N + nP + 1];
    Q0[c] = A.x[c * A.N + nQ];
    Q1[c] = A.x[c * A.N + nQ + 1];
  }
  double s, u;
  closest(P0, P1, Q0, Q1, s, u);
  double dvec[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) dvec[c] = (P0[c] + s * (P1[c] - P0[c])) - (Q0[c] + u * (Q1[c] - Q0[c]));
  const double d2 = dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2];
  if (!(d2 > 0.0)) return out;
  const double id = rsqrt(d2);              // 1 / d
  const double d = d2 * id;
  const double delta = (rada + radb) - d;
  if (!(delta > 0.0)) return out;
  const double nrm[3] = {dvec[0] * id, dvec[1] * id, dvec[2] * id};
  double vrel = 0.0, vr[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double vp0 = A.v[c * A.N + nP], vp1 = A.v[c * A.N + nP + 1];
    const double vq0 = A.v[c * A.N + nQ], vq1 = A.v[c * A.N + nQ + 1];
    vr[c] = ((1.0 - s) * vp0 + s * vp1) - ((1.0 - u) * vq0 + u * vq1);
    vrel += vr[c] * nrm[c];
  }
  double fmag = A.k * delta - A.c * vrel;
  if (fmag < 0.0) fmag = 0.0;
  // friction: -mu fmag v_t / max(|v_t|, v_slip) with v_t the tangential relative velocity
  double ft[3] = {0.0, 0.0, 0.0};
  if (A.mu > 0.0 && fmag > 0.0) {
    double vt[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) vt[c] = vr[c] - vrel * nrm[c];
    // 1 / max(|v_t|, v_slip) = min(1 / |v_t|, 1 / v_slip)
    const double sp2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
    const double fr = -A.mu * fmag * fmin(rsqrt(sp2), A.inv_vslip);
#pragma unroll
    for (int c = 0; c < 3; ++c) ft[c] = fr * vt[c];
  }
  // force on the first segment of the pair is +(fmag n + ft), on the second the opposite
  const double wa = first ? (1.0 - s) : -(1.0 - u);
  const double wb = first ? s : -u;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double fc = fmag * nrm[c] + ft[c];
    out.fa[c] = wa * fc;
    out.fb[c] = wb * fc;
  }
  out.hit = true;
  return out;
}

// FP32 lower bounds of the distance of segments a and b (midpoints m, half lengths h, half
// edges e) against touch = r_a + r_b + extra + tol, tol covering the rounding of the FP32
// inputs and of these expressions: false when the pair is certainly farther apart.
__device__ __forceinline__ bool may_touch(float4 ga, float4 gb, float4 ea, float4 eb, float touch_base) {
  const float ddx = ga.x - gb.x, ddy = ga.y - gb.y, ddz = ga.z - gb.z;
  const float dm2 = ddx * ddx + ddy * ddy + ddz * ddz;
  const float ma_inf = fmaxf(fabsf(ga.x), fmaxf(fabsf(ga.y), fabsf(ga.z)));
  const float mb_inf = fmaxf(fabsf(gb.x), fmaxf(fabsf(gb.y), fabsf(gb.z)));
  const float touch = touch_base + 1e-6f + 4e-6f * (ma_inf + mb_inf + ga.w + gb.w);
  const float reach = touch + ga.w + gb.w;
  if (dm2 > reach * reach) return false;
  // separating axis along m_a - m_b: |dm| - (|e_a . dm| + |e_b . dm|) / |dm| > touch
  const float pa = fabsf(ea.x * ddx + ea.y * ddy + ea.z * ddz);
  const float pb = fabsf(eb.x * ddx + eb.y * ddy + eb.z * ddz);
  return !(dm2 > 0.f && dm2 - (pa + pb) > touch * sqrtf(dm2));
}

// Calls visit(b, rb) for every segment b of another rod in the 27-cell neighbourhood of slot q
// (cell-ordered records) that may come within r_a + r_b + extra of the slot's segment, in list
// order.  The three cells of each (y, z) row are consecutive in the list and scanned as one
// range; the next candidate's records are loaded while the current one is tested.
template <class Visit>
__device__ __forceinline__ void scan_neighbourhood(const ContactArgs& A, int64_t q, float extra, Visit& visit) {
  const float4 ga = A.recA[q];
  const int4 ba = A.recB[q];
  const float4 ea = A.recC[q];
  const int ra = ba.y;
  const float rada = __int_as_float(ba.z);
  const int cell = A.seg_cell[ba.x];
  const int cx = cell % A.dim[0], cy = (cell / A.dim[0]) % A.dim[1], cz = cell / (A.dim[0] * A.dim[1]);
  const int x0 = max(cx - 1, 0), x1 = min(cx + 1, A.dim[0] - 1);
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= A.dim[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = cy + dy;
      if (y < 0 || y >= A.dim[1]) continue;
      const int row = (z * A.dim[1] + y) * A.dim[0];
      const int b0 = A.cell_start[row + x0], b1 = A.cell_start[row + x1 + 1];
      if (b1 - b0 > 3 * kCellCap) {
        atomicOr(A.err, ERR_OVERFLOW);
        continue;
      }
      int4 bb_next = make_int4(0, 0, 0, 0);
      float4 gb_next = make_float4(0.f, 0.f, 0.f, 0.f);
      if (b0 < b1) {
        bb_next = A.recB[b0];
        gb_next = A.recA[b0];
      }
      for (int t = b0; t < b1;) {
        const int tc = t;
        const int4 bb = bb_next;
        const float4 gb = gb_next;
        t = (bb.y == ra) ? bb.w : t + 1;  // own rod: skip its run in this cell
        if (t < b1) {
          bb_next = A.recB[t];
          gb_next = A.recA[t];
        }
        if (bb.y == ra) continue;
        if (!may_touch(ga, gb, ea, A.recC[tc], rada + __int_as_float(bb.z) + extra)) continue;
        visit(bb.x, bb.y);
      }
    }
  }
}

struct ForceSum {
  const ContactArgs& A;
  int a, ra;
  double fa[3], fb[3];
  __device__ ForceSum(const ContactArgs& args, int a_, int ra_) : A(args), a(a_), ra(ra_) {
#pragma unroll
    for (int c = 0; c < 3; ++c) fa[c] = fb[c] = 0.0;
  }
  __device__ void operator()(int b, int rb) {
    const PairForce pf = pair_force(A, a, ra, b, rb);
    if (pf.hit) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fa[c] += pf.fa[c];
        fb[c] += pf.fb[c];
      }
    }
  }
  __device__ void store(double* fseg, int64_t E) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fseg[c * E + a] = fa[c];
      fseg[(3 + c) * E + a] = fb[c];
    }
  }
};

// Contact forces on the two nodes of segment a from its skin list: candidates culled in FP32
// against the segment proxies of the current positions (written by the step kernel that
// produced them) and evaluated in FP64; a segment whose list overflowed scans its
// neighbourhood of the last build with the skin bound (the build's records are stale by less
// than skin / 2 per node, which the skin covers).
__device__ __forceinline__ void listed_forces(const ContactArgs& A, int64_t a, ForceSum& f) {
  const int n = A.nbr_count[a];
  if (n <= kNbrCap) {
    if (n > 0) {
      static_assert(kNbrCap <= 32, "the survivors of the cull are kept in a 32-bit mask");
      // pass 1: FP32 cull of every candidate (groups of four: all indices, then all proxies, so
      // that four independent loads are in flight); survivors go to a bit mask
      const float4 ga = A.seg_prox[2 * a], ea = A.seg_prox[2 * a + 1];
      unsigned hit = 0u;
      constexpr int kG = 4;
      for (int k0 = 0; k0 < n; k0 += kG) {
        int bs[kG];
        float4 gb[kG], eb[kG];
#pragma unroll
        for (int t = 0; t < kG; ++t) bs[t] = (k0 + t < n) ? A.nbr[(k0 + t) * A.E + a] : -1;
#pragma unroll
        for (int t = 0; t < kG; ++t) {
          if (bs[t] >= 0) {
            gb[t] = A.seg_prox[2 * (int64_t)bs[t]];
            eb[t] = A.seg_prox[2 * (int64_t)bs[t] + 1];
          }
        }
#pragma unroll
        for (int t = 0; t < kG; ++t)
          if (bs[t] >= 0 && may_touch(ga, gb[t], ea, eb[t], ea.w + eb[t].w)) hit |= 1u << (k0 + t);
      }
      // pass 2: FP64 evaluation of the survivors in list order
      while (hit) {
        const int k = __ffs(hit) - 1;
        hit &= hit - 1;
        const int b = A.nbr[k * A.E + a];
        f(b, A.seg_rod[b]);
      }
    }
  } else {
    scan_neighbourhood(A, A.slot_of[a], A.skin, f);
  }
}

}  // namespace
}  // namespace rod
