// Checks that the FP32 contact cull of rod_cull.h never rejects a pair of FP64 segments that
// touch (exact distance below r_a + r_b, or below r_a + r_b + skin for a list build): random
// pairs with coordinates up to 1.2 m, half lengths 2e-4..1e-2 m, radii 1e-4..3e-3 m, a third of
// them nearly parallel (angles down to 1e-7 rad), most placed near the touching distance.  The
// FP32 proxies are formed as the library forms them: the step kernel's (midpoint and half edge
// of the FP32-rounded end points) and the cell records' (half edge rounded from FP64).  The
// reference distance is the minimum of the squared distance over the unit square in long
// double: the interior critical point when it lies inside, else the four end-point-to-segment
// distances.
// Prints "<pairs> <violations> <far pairs> <far pairs passed by bound 1> <far pairs passed by both>"
// (far: exact distance above 2 (r_a + r_b + skin)) and exits 0.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "../../paper_2605_13766_gb300/csrc/rod_cull.h"

using LD = long double;

static uint64_t s = 0x243F6A8885A308D3ull;
static uint64_t next() {  // xorshift64*
  s ^= s >> 12;
  s ^= s << 25;
  s ^= s >> 27;
  return s * 0x2545F4914F6CDD1Dull;
}
static double uni() { return (next() >> 11) * 0x1p-53; }
static double uni(double a, double b) { return a + (b - a) * uni(); }
static double logu(double a, double b) { return std::exp(uni(std::log(a), std::log(b))); }

static void unit(double u[3]) {
  double n;
  do {
    for (int c = 0; c < 3; ++c) u[c] = uni(-1.0, 1.0);
    n = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  } while (n < 0.1 || n > 1.0);
  for (int c = 0; c < 3; ++c) u[c] /= n;
}

static LD dot(const LD a[3], const LD b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static LD point_segment(const LD p[3], const LD q0[3], const LD q1[3]) {
  LD d[3], r[3];
  for (int c = 0; c < 3; ++c) {
    d[c] = q1[c] - q0[c];
    r[c] = p[c] - q0[c];
  }
  const LD dd = dot(d, d);
  LD t = dd > 0 ? dot(r, d) / dd : 0;
  t = t < 0 ? 0 : (t > 1 ? 1 : t);
  LD w[3];
  for (int c = 0; c < 3; ++c) w[c] = r[c] - t * d[c];
  return std::sqrt(dot(w, w));
}

static LD segment_distance(const double a0[3], const double a1[3], const double b0[3], const double b1[3]) {
  LD A0[3], A1[3], B0[3], B1[3];
  for (int c = 0; c < 3; ++c) {
    A0[c] = a0[c];
    A1[c] = a1[c];
    B0[c] = b0[c];
    B1[c] = b1[c];
  }
  LD d = point_segment(A0, B0, B1);
  LD t = point_segment(A1, B0, B1);
  if (t < d) d = t;
  t = point_segment(B0, A0, A1);
  if (t < d) d = t;
  t = point_segment(B1, A0, A1);
  if (t < d) d = t;
  LD d1[3], d2[3], r[3];
  for (int c = 0; c < 3; ++c) {
    d1[c] = A1[c] - A0[c];
    d2[c] = B1[c] - B0[c];
    r[c] = A0[c] - B0[c];
  }
  const LD a = dot(d1, d1), e = dot(d2, d2), b = dot(d1, d2), cc = dot(d1, r), f = dot(d2, r);
  const LD den = a * e - b * b;
  if (den > 0) {
    const LD sp = (b * f - cc * e) / den, u = (a * f - b * cc) / den;
    if (sp > 0 && sp < 1 && u > 0 && u < 1) {
      LD w[3];
      for (int c = 0; c < 3; ++c) w[c] = r[c] + sp * d1[c] - u * d2[c];
      const LD di = std::sqrt(dot(w, w));
      if (di < d) d = di;
    }
  }
  return d;
}

// the step kernel's proxy: FP32 end points, midpoint and half edge from them, half length
static void step_proxy(const double p0[3], const double p1[3], float radius, rod::float4& g, rod::float4& e) {
  float f0[3], f1[3], he[3];
  for (int c = 0; c < 3; ++c) {
    f0[c] = static_cast<float>(p0[c]);
    f1[c] = static_cast<float>(p1[c]);
    he[c] = 0.5f * (f1[c] - f0[c]);
  }
  const float hl = std::sqrt(std::fma(he[0], he[0], std::fma(he[1], he[1], he[2] * he[2])));
  g = {0.5f * (f0[0] + f1[0]), 0.5f * (f0[1] + f1[1]), 0.5f * (f0[2] + f1[2]), hl};
  e = {he[0], he[1], he[2], radius};
}

// the cell records' half edge (rounded from the FP64 difference)
static rod::float4 record_edge(const double p0[3], const double p1[3]) {
  return {static_cast<float>(0.5 * (p1[0] - p0[0])), static_cast<float>(0.5 * (p1[1] - p0[1])),
          static_cast<float>(0.5 * (p1[2] - p0[2])), 0.f};
}

// the first bound alone (the cull before the line-distance bound), for the efficacy count
static bool bound1_passes(rod::float4 ga, rod::float4 gb, rod::float4 ea, rod::float4 eb, float touch_base) {
  const float ddx = ga.x - gb.x, ddy = ga.y - gb.y, ddz = ga.z - gb.z;
  const float dm2 = ddx * ddx + ddy * ddy + ddz * ddz;
  const float ma = std::fmax(std::fabs(ga.x), std::fmax(std::fabs(ga.y), std::fabs(ga.z)));
  const float mb = std::fmax(std::fabs(gb.x), std::fmax(std::fabs(gb.y), std::fabs(gb.z)));
  const float touch = touch_base + 1e-6f + 4e-6f * (ma + mb + ga.w + gb.w);
  const float reach = touch + ga.w + gb.w;
  if (dm2 > reach * reach) return false;
  const float pa = std::fabs(ea.x * ddx + ea.y * ddy + ea.z * ddz);
  const float pb = std::fabs(eb.x * ddx + eb.y * ddy + eb.z * ddz);
  return !(dm2 > 0.f && dm2 - (pa + pb) > touch * std::sqrt(dm2));
}

int main() {
  const long n_pairs = 2000000;
  long violations = 0, far = 0, far_b1 = 0, far_both = 0;
  for (long i = 0; i < n_pairs; ++i) {
    double ua[3], ub[3], w[3], ma[3];
    unit(ua);
    for (int c = 0; c < 3; ++c) ma[c] = uni(-1.2, 1.2);
    const double ha = logu(2e-4, 1e-2), hb = logu(2e-4, 1e-2);
    const double ra = uni(1e-4, 3e-3), rb = uni(1e-4, 3e-3);
    const double skin = (next() & 1) ? 5e-4 : 0.0;
    const double touch = ra + rb + skin;
    // direction of b: nearly parallel to a (a third), else random
    if (next() % 3 == 0) {
      double q[3];
      unit(q);
      const double ang = logu(1e-7, 0.1);
      double n = 0;
      for (int c = 0; c < 3; ++c) {
        ub[c] = ua[c] + ang * q[c];
        n += ub[c] * ub[c];
      }
      n = std::sqrt(n);
      for (int c = 0; c < 3; ++c) ub[c] /= n;
    } else {
      unit(ub);
    }
    // b's midpoint: a point near segment a (parameter beyond the ends at times), moved off by
    // about the touching distance in a random direction, and slid along b
    unit(w);
    const double sa = uni(-1.4, 1.4), sb = uni(-1.4, 1.4);
    const double off = (next() % 4 == 0) ? uni(0.0, 4.0 * (touch + ha + hb)) : touch * uni(0.3, 3.0);
    double mb[3];
    for (int c = 0; c < 3; ++c) mb[c] = ma[c] + sa * ha * ua[c] + off * w[c] - sb * hb * ub[c];
    double a0[3], a1[3], b0[3], b1[3];
    for (int c = 0; c < 3; ++c) {
      a0[c] = ma[c] - ha * ua[c];
      a1[c] = ma[c] + ha * ua[c];
      b0[c] = mb[c] - hb * ub[c];
      b1[c] = mb[c] + hb * ub[c];
    }
    const LD d = segment_distance(a0, a1, b0, b1);
    const float touch_base = static_cast<float>(ra) + static_cast<float>(rb) + static_cast<float>(skin);
    rod::float4 ga, ea, gb, eb;
    step_proxy(a0, a1, static_cast<float>(ra), ga, ea);
    step_proxy(b0, b1, static_cast<float>(rb), gb, eb);
    const bool pass_step = rod::may_touch(ga, gb, ea, eb, touch_base);
    const bool pass_rec = rod::may_touch(ga, gb, record_edge(a0, a1), record_edge(b0, b1), touch_base);
    if (d < static_cast<LD>(touch) && !(pass_step && pass_rec)) {
      if (violations < 10)
        std::fprintf(stderr, "violation: d = %.17Lg touch = %.17g step %d records %d\n", d, touch, pass_step, pass_rec);
      ++violations;
    }
    if (d > 2.0L * static_cast<LD>(touch)) {
      ++far;
      if (bound1_passes(ga, gb, ea, eb, touch_base)) ++far_b1;
      if (pass_step) ++far_both;
    }
  }
  std::printf("%ld %ld %ld %ld %ld\n", n_pairs, violations, far, far_b1, far_both);
  return 0;
}
