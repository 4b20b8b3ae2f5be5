/*
 * oracle_ad.cpp -- the oracle's own source (rod_oracle.c) compiled over two other number types.
 *
 * TEST INFRASTRUCTURE ONLY (tests and the script that counts the method's operations).
 *
 *   orc_dual:  forward-mode dual numbers (value, tangent).  Every elementary operation carries
 *              its exact derivative, so a run of orc_step gives the Jacobian-vector product of
 *              the oracle's discrete step map (the tangent of the same function the oracle
 *              evaluates, branches included) with no difference quotient anywhere.  This is
 *              the directional derivative that a reverse (adjoint) sweep of the same steps
 *              must reproduce: g . u = d/dh L(p + h u) at h = 0.
 *   orc_count: numbers that count every FP64 addition/subtraction, multiplication, division
 *              and special-function call made on them, so a run of orc_step counts the
 *              method's arithmetic per element-step as the oracle states it.
 *
 * The source is included unchanged: `double` is redefined to the number type around the
 * inclusion, inside a namespace of its own (the header's ORC_CXX_LINKAGE gives the functions
 * C++ linkage there).  The exported entry points below take plain doubles.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "rod_oracle.h"

/* ------------------------------------------------------------------ dual numbers */

struct Dual {
  double v, d;
  Dual() = default;
  Dual(double x) : v(x), d(0.0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
  explicit operator int64_t() const { return static_cast<int64_t>(v); }
  explicit operator int() const { return static_cast<int>(v); }
  Dual& operator+=(const Dual& b) { d += b.d; v += b.v; return *this; }
  Dual& operator-=(const Dual& b) { d -= b.d; v -= b.v; return *this; }
  Dual& operator*=(const Dual& b) { *this = Dual(v * b.v, d * b.v + v * b.d); return *this; }
  Dual& operator/=(const Dual& b) {
    const double q = v / b.v;
    *this = Dual(q, (d - q * b.d) / b.v);
    return *this;
  }
};
static inline Dual operator+(Dual a, const Dual& b) { return a += b; }
static inline Dual operator-(Dual a, const Dual& b) { return a -= b; }
static inline Dual operator*(Dual a, const Dual& b) { return a *= b; }
static inline Dual operator/(Dual a, const Dual& b) { return a /= b; }
static inline Dual operator-(const Dual& a) { return Dual(-a.v, -a.d); }
static inline Dual operator+(const Dual& a) { return a; }
static inline bool operator<(const Dual& a, const Dual& b) { return a.v < b.v; }
static inline bool operator>(const Dual& a, const Dual& b) { return a.v > b.v; }
static inline bool operator<=(const Dual& a, const Dual& b) { return a.v <= b.v; }
static inline bool operator>=(const Dual& a, const Dual& b) { return a.v >= b.v; }
static inline bool operator==(const Dual& a, const Dual& b) { return a.v == b.v; }
static inline bool operator!=(const Dual& a, const Dual& b) { return a.v != b.v; }
/* d sqrt(x) = dx / (2 sqrt x); at x = 0 the tangent is taken as 0 (the oracle only takes the
 * root of sums of squares, whose tangent vanishes there) */
static inline Dual sqrt(const Dual& a) {
  const double s = sqrt(a.v);
  return Dual(s, s > 0.0 ? a.d / (2.0 * s) : 0.0);
}
static inline Dual sin(const Dual& a) { return Dual(sin(a.v), cos(a.v) * a.d); }
static inline Dual cos(const Dual& a) { return Dual(cos(a.v), -sin(a.v) * a.d); }
/* d atan2(y, x) = (x dy - y dx) / (x^2 + y^2) */
static inline Dual atan2(const Dual& y, const Dual& x) {
  const double r2 = x.v * x.v + y.v * y.v;
  return Dual(atan2(y.v, x.v), r2 > 0.0 ? (x.v * y.d - y.v * x.d) / r2 : 0.0);
}
static inline Dual floor(const Dual& a) { return Dual(floor(a.v), 0.0); }
static inline Dual fabs(const Dual& a) { return a.v < 0.0 ? -a : a; }
static inline bool isfinite(const Dual& a) { return std::isfinite(a.v) && std::isfinite(a.d); }

/* ------------------------------------------------------------------ counting numbers */

/* counters: additions and subtractions, multiplications, divisions, square roots, sin and
 * cos, atan2, floor, fabs */
enum { C_ADD, C_MUL, C_DIV, C_SQRT, C_SINCOS, C_ATAN2, C_FLOOR, C_FABS, C_NUM };
static int64_t g_count[C_NUM];

struct Counted {
  double v;
  Counted() = default;
  Counted(double x) : v(x) {}
  explicit operator int64_t() const { return static_cast<int64_t>(v); }
  explicit operator int() const { return static_cast<int>(v); }
  Counted& operator+=(const Counted& b) { ++g_count[C_ADD]; v += b.v; return *this; }
  Counted& operator-=(const Counted& b) { ++g_count[C_ADD]; v -= b.v; return *this; }
  Counted& operator*=(const Counted& b) { ++g_count[C_MUL]; v *= b.v; return *this; }
  Counted& operator/=(const Counted& b) { ++g_count[C_DIV]; v /= b.v; return *this; }
};
static inline Counted operator+(Counted a, const Counted& b) { return a += b; }
static inline Counted operator-(Counted a, const Counted& b) { return a -= b; }
static inline Counted operator*(Counted a, const Counted& b) { return a *= b; }
static inline Counted operator/(Counted a, const Counted& b) { return a /= b; }
static inline Counted operator-(const Counted& a) { return Counted(-a.v); }  /* a sign flip, not counted */
static inline Counted operator+(const Counted& a) { return a; }
static inline bool operator<(const Counted& a, const Counted& b) { return a.v < b.v; }
static inline bool operator>(const Counted& a, const Counted& b) { return a.v > b.v; }
static inline bool operator<=(const Counted& a, const Counted& b) { return a.v <= b.v; }
static inline bool operator>=(const Counted& a, const Counted& b) { return a.v >= b.v; }
static inline bool operator==(const Counted& a, const Counted& b) { return a.v == b.v; }
static inline bool operator!=(const Counted& a, const Counted& b) { return a.v != b.v; }
static inline Counted sqrt(const Counted& a) { ++g_count[C_SQRT]; return Counted(sqrt(a.v)); }
static inline Counted sin(const Counted& a) { ++g_count[C_SINCOS]; return Counted(sin(a.v)); }
static inline Counted cos(const Counted& a) { ++g_count[C_SINCOS]; return Counted(cos(a.v)); }
static inline Counted atan2(const Counted& y, const Counted& x) { ++g_count[C_ATAN2]; return Counted(atan2(y.v, x.v)); }
static inline Counted floor(const Counted& a) { ++g_count[C_FLOOR]; return Counted(floor(a.v)); }
static inline Counted fabs(const Counted& a) { ++g_count[C_FABS]; return Counted(fabs(a.v)); }
static inline bool isfinite(const Counted& a) { return std::isfinite(a.v); }

/* ------------------------------------------------------------------ the oracle, twice */

#define ORC_CXX_LINKAGE
namespace orc_dual {
#undef ROD_ORACLE_H
#define double Dual
#include "rod_oracle.c"
#undef double
}  // namespace orc_dual

namespace orc_count {
#undef ROD_ORACLE_H
#define double Counted
#include "rod_oracle.c"
#undef double
}  // namespace orc_count

/* ------------------------------------------------------------------ parameter conversion */

static inline Dual make_num(double v, double d, Dual*) { return Dual(v, d); }
static inline Counted make_num(double v, double, Counted*) { return Counted(v); }

/* Arrays of number type T holding the parameters (kept alive for the call). */
template <class T>
struct Store {
  std::vector<std::vector<T>> keep;
  /* n values from a (zeros if a is NULL) with tangents tan (zeros if NULL) */
  const T* arr(const double* a, int64_t n, const double* tan = nullptr) {
    keep.emplace_back(static_cast<size_t>(n > 0 ? n : 1));
    std::vector<T>& out = keep.back();
    for (int64_t i = 0; i < n; ++i)
      out[i] = make_num(a ? a[i] : 0.0, tan ? tan[i] : 0.0, static_cast<T*>(nullptr));
    return out.data();
  }
  const T* opt(const double* a, int64_t n, const double* tan = nullptr) {
    return (a || tan) ? arr(a, n, tan) : nullptr;
  }
};

/* Copy of the plain parameters p over number type T; the rest curvature and the element couples
 * get the tangents d_kappa [3V] and d_couple [3E] (NULL: zero). */
template <class T, class PT>
static void convert_params(const orc_params* p, PT* q, Store<T>& st, const double* d_kappa,
                           const double* d_couple) {
  const int64_t R = p->n_rods;
  int64_t E = 0;
  for (int64_t r = 0; r < R; ++r) E += p->n_elem[r];
  const int64_t V = E - R, W = p->n_walls;
  memset(static_cast<void*>(q), 0, sizeof *q);
  q->n_rods = p->n_rods;
  q->n_elem = p->n_elem;
  q->rest_len = st.arr(p->rest_len, E);
  q->radius = st.arr(p->radius, R);
  q->youngs = st.arr(p->youngs, R);
  q->shear_mod = st.arr(p->shear_mod, R);
  q->density = st.arr(p->density, R);
  q->alpha_c = p->alpha_c;
  q->clamp_base = p->clamp_base;
  q->rest_kappa = st.opt(p->rest_kappa, 3 * V, d_kappa);
  q->rest_sigma = st.opt(p->rest_sigma, 3 * E);
  for (int c = 0; c < 3; ++c) q->gravity[c] = p->gravity[c];
  q->nu_damp = p->nu_damp;
  q->stokes_gamma = p->stokes_gamma;
  q->tip_force = st.opt(p->tip_force, 3 * R);
  q->act_amp = st.opt(p->act_amp, R);
  q->act_period = st.opt(p->act_period, R);
  q->act_phase = st.opt(p->act_phase, R);
  q->elem_couple = st.opt(p->elem_couple, 3 * E, d_couple);
  q->contact = p->contact;
  q->contact_k = p->contact_k;
  q->contact_c = p->contact_c;
  q->cell_size = p->cell_size;
  q->broad_phase = p->broad_phase;
  q->magnetization = st.opt(p->magnetization, 3 * E);
  for (int c = 0; c < 3; ++c) {
    q->field_b0[c] = p->field_b0[c];
    q->field_bc[c] = p->field_bc[c];
    q->field_bs[c] = p->field_bs[c];
  }
  q->field_omega = p->field_omega;
  q->muscle_amp = st.opt(p->muscle_amp, R);
  q->muscle_period = st.opt(p->muscle_period, R);
  q->muscle_wavelength = st.opt(p->muscle_wavelength, R);
  q->muscle_phase = st.opt(p->muscle_phase, R);
  q->contact_mu = p->contact_mu;
  q->contact_vslip = p->contact_vslip;
  q->n_walls = p->n_walls;
  q->wall_point = st.opt(p->wall_point, 3 * W);
  q->wall_normal = st.opt(p->wall_normal, 3 * W);
  q->wall_velocity = st.opt(p->wall_velocity, 3 * W);
  q->wall_k = p->wall_k;
  q->wall_c = p->wall_c;
  q->wall_mu = p->wall_mu;
  q->wall_vslip = p->wall_vslip;
}

static int64_t count_elems(const orc_params* p) {
  int64_t E = 0;
  for (int r = 0; r < p->n_rods; ++r) E += p->n_elem[r];
  return E;
}

/* ------------------------------------------------------------------ exported entry points */

extern "C" {

/* Jacobian-vector product of n_steps oracle steps: the state (x, v [3N], Q [9E], w [3E]) is
 * advanced in place exactly as orc_step advances it, and the tangents (dx, dv, dQ, dw, same
 * layout) are advanced with it; d_rest_kappa [3V] and d_elem_couple [3E] are the tangents of
 * the rest curvature and the element couples (NULL: zero).  Returns 0, or -1 (message from
 * orcd_last_error). */
int orcd_step_jvp(const orc_params* p, double t, double dt, int64_t n_steps, double* x, double* v, double* Q,
                  double* w, double* dx, double* dv, double* dQ, double* dw, const double* d_rest_kappa,
                  const double* d_elem_couple) {
  Store<Dual> st;
  orc_dual::orc_params q;
  convert_params<Dual>(p, &q, st, d_rest_kappa, d_elem_couple);
  const int64_t E = count_elems(p), N = E + p->n_rods;
  std::vector<Dual> X(3 * N), Vv(3 * N), QQ(9 * E), Ww(3 * E);
  for (int64_t i = 0; i < 3 * N; ++i) {
    X[i] = Dual(x[i], dx[i]);
    Vv[i] = Dual(v[i], dv[i]);
  }
  for (int64_t i = 0; i < 9 * E; ++i) QQ[i] = Dual(Q[i], dQ[i]);
  for (int64_t i = 0; i < 3 * E; ++i) Ww[i] = Dual(w[i], dw[i]);
  const int rc = orc_dual::orc_step(&q, Dual(t), Dual(dt), n_steps, X.data(), Vv.data(), QQ.data(), Ww.data());
  for (int64_t i = 0; i < 3 * N; ++i) {
    x[i] = X[i].v, dx[i] = X[i].d;
    v[i] = Vv[i].v, dv[i] = Vv[i].d;
  }
  for (int64_t i = 0; i < 9 * E; ++i) Q[i] = QQ[i].v, dQ[i] = QQ[i].d;
  for (int64_t i = 0; i < 3 * E; ++i) w[i] = Ww[i].v, dw[i] = Ww[i].d;
  return rc;
}

const char* orcd_last_error(void) { return orc_dual::orc_last_error(); }

/* n_steps oracle steps (state advanced in place as orc_step does) counting the FP64 work:
 * counts[0..7] receive the additions and subtractions, multiplications, divisions, square
 * roots, sin and cos calls, atan2 calls, floor calls and fabs calls made. */
int orcc_step_count(const orc_params* p, double t, double dt, int64_t n_steps, double* x, double* v, double* Q,
                    double* w, int64_t* counts) {
  Store<Counted> st;
  orc_count::orc_params q;
  convert_params<Counted>(p, &q, st, nullptr, nullptr);
  const int64_t E = count_elems(p), N = E + p->n_rods;
  std::vector<Counted> X(3 * N), Vv(3 * N), QQ(9 * E), Ww(3 * E);
  for (int64_t i = 0; i < 3 * N; ++i) X[i] = Counted(x[i]), Vv[i] = Counted(v[i]);
  for (int64_t i = 0; i < 9 * E; ++i) QQ[i] = Counted(Q[i]);
  for (int64_t i = 0; i < 3 * E; ++i) Ww[i] = Counted(w[i]);
  for (int k = 0; k < C_NUM; ++k) g_count[k] = 0;
  const int rc = orc_count::orc_step(&q, Counted(t), Counted(dt), n_steps, X.data(), Vv.data(), QQ.data(), Ww.data());
  for (int k = 0; k < C_NUM; ++k) counts[k] = g_count[k];
  for (int64_t i = 0; i < 3 * N; ++i) x[i] = X[i].v, v[i] = Vv[i].v;
  for (int64_t i = 0; i < 9 * E; ++i) Q[i] = QQ[i].v;
  for (int64_t i = 0; i < 3 * E; ++i) w[i] = Ww[i].v;
  return rc;
}

const char* orcc_last_error(void) { return orc_count::orc_last_error(); }

}  /* extern "C" */
