/*
 * rod_oracle.c -- plain FP64 CPU oracle of the discrete Cosserat-rod step.
 *
 * TEST INFRASTRUCTURE ONLY (tests, the package smoke check and the benchmark's CPU
 * baseline).  Deliberately plain: scalar loops, whole-system temporaries, no blocking,
 * no fusion, no reordering beyond what the definitions state.  Compiled with
 * -O2 -ffp-contract=off so that every product and sum is rounded as written.
 *
 * Notation (per rod with n elements): nodes j = 0..n, elements i = 0..n-1,
 * Voronoi points k = 0..n-2 (between elements k and k+1).
 *   l_i = x_{i+1} - x_i, ell_i = |l_i|, e_i = ell_i / rl_i  (rl = rest length)
 *   sigma_i = Q_i l_i / rl_i - (0,0,1)        [= Q(e t - d3), sigma = Q(r' - d3), Methods]
 *   kappa_k = -ax(log(Q_{k+1} Q_k^T)) / D_k   [kappa = ax(Q dQ^T/ds), Methods]
 *   D_k = (rl_k + rl_{k+1})/2, eps_k = (ell_k + ell_{k+1}) / (rl_k + rl_{k+1})
 *   n_i = S(sigma_i - sigma0_i),  N_i = Q_i^T n_i / e_i   (lab frame, Eq. 1a)
 *   F_j = N_j - N_{j-1}, with N_{-1} = N_n = 0          (difference operator, Eq. 1a)
 *   m_k = B(kappa_k - kappa0_k); P_k = m_k / eps_k^3; T_k = (kappa_k x m_k) D_k / eps_k^3
 *   tau_b_i = P_i - P_{i-1} + (T_{i-1} + T_i)/2, ghosts P,T at k = -1, n-1 are zero (Eq. 1b,
 *             first two terms: difference and trapezoidal averaging operators)
 *   tau_s_i = ((Q_i t_i) x n_i) rl_i                     (Eq. 1b, shear term; t = unit tangent)
 *   tau_u_i = (J_i w_i / e_i) x w_i + (J_i w_i / e_i^2) de_i/dt,
 *             de_i/dt = t_i . (v_{i+1} - v_i) / rl_i    (Eq. 1b, last transport terms)
 *   J_i = rho rl_i diag(I1, I2, I1+I2); lumped node mass m_j = (M_{j-1} + M_j)/2, M_i = rho A rl_i
 *   a_j = (F_j + f_j) / m_j;  dw_i/dt = e_i J_i^{-1} (tau_b + tau_s + tau_u + c)_i   (Eq. 1)
 * Time stepping: position Verlet (half kinematic stage, dynamic stage at t + dt/2, half
 * kinematic stage), kinematic constraints after every stage (Results, performance section).
 * Director update: Q <- exp(-h [w]x) Q, which is the exact flow of dQ/dt = -[w]x Q, i.e. of
 * w = ax(Q dQ^T/dt) (Methods) for w held constant over the stage.
 *
 * Readings where the paper is silent (all mirrored in the design notes):
 *   - rho is a volumetric density (kg/m^3), line density rho*A;
 *   - the tangent "t" of the shear couple is the unit tangent l/ell;
 *   - linear damping with one decay rate nu/(rho A) for translation and rotation:
 *     force -nu*rlN_j*v_j (rlN_j = nodal rest length share), couple -nu*rl_i*(I_c/A)*w_ic;
 *     Stokes drag: force -gamma*rlN_j*v_j (no rotational drag); both use the velocities at
 *     the start of the dynamic stage;
 *   - the base actuation couple A sin(2 pi t/T + phi) d1 acts on the first element not held
 *     by a clamp (element 1 of a clamped rod, element 0 otherwise);
 *   - contact: pair of segments of different rods, closest points by the clamped
 *     two-parameter minimisation, overlap delta = r_a + r_b - d, force magnitude
 *     max(0, k delta - c v_rel.n) along n = (p_a - p_b)/d, split (1-s, s) onto the segment
 *     nodes; the lower segment index is always the first segment of the pair; d == 0 gives
 *     no force; no contact couples.
 */
#include "rod_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static char g_err[512];

static int fail(const char* msg) {
  snprintf(g_err, sizeof g_err, "%s", msg);
  return -1;
}
const char* orc_last_error(void) { return g_err; }

/* ---------------------------------------------------------------- sizes / offsets */

int64_t orc_num_elems(const orc_params* p) {
  int64_t s = 0;
  for (int r = 0; r < p->n_rods; ++r) s += p->n_elem[r];
  return s;
}
int64_t orc_num_nodes(const orc_params* p) { return orc_num_elems(p) + p->n_rods; }
int64_t orc_num_voronoi(const orc_params* p) { return orc_num_elems(p) - p->n_rods; }

typedef struct {
  int64_t node0, elem0, vor0; /* first node / element / Voronoi index of the rod */
  int n;                      /* elements */
} rod_range;

/* ranges of every rod, in CSR order (caller frees) */
static rod_range* rod_ranges(const orc_params* p) {
  rod_range* g = (rod_range*)malloc(sizeof(rod_range) * (size_t)p->n_rods);
  if (!g) return NULL;
  int64_t node0 = 0, elem0 = 0, vor0 = 0;
  for (int r = 0; r < p->n_rods; ++r) {
    g[r].node0 = node0;
    g[r].elem0 = elem0;
    g[r].vor0 = vor0;
    g[r].n = p->n_elem[r];
    node0 += p->n_elem[r] + 1;
    elem0 += p->n_elem[r];
    vor0 += p->n_elem[r] - 1;
  }
  return g;
}

/* ---------------------------------------------------------------- small vector helpers */

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double c[3]) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static void ld3(const double* arr, int64_t n, int64_t i, double o[3]) {
  for (int c = 0; c < 3; ++c) o[c] = arr[c * n + i];
}
static void st3(double* arr, int64_t n, int64_t i, const double o[3]) {
  for (int c = 0; c < 3; ++c) arr[c * n + i] = o[c];
}
static void acc3(double* arr, int64_t n, int64_t i, const double o[3], double scale) {
  for (int c = 0; c < 3; ++c) arr[c * n + i] += scale * o[c];
}
static void ldQ(const double* Q, int64_t E, int64_t i, double M[9]) {
  for (int a = 0; a < 9; ++a) M[a] = Q[a * E + i];
}
static void stQ(double* Q, int64_t E, int64_t i, const double M[9]) {
  for (int a = 0; a < 9; ++a) Q[a * E + i] = M[a];
}
/* local = Q lab:  o_a = sum_b Q_ab v_b  (rows of Q are the directors) */
static void mat_vec(const double M[9], const double v[3], double o[3]) {
  for (int a = 0; a < 3; ++a) o[a] = M[3 * a + 0] * v[0] + M[3 * a + 1] * v[1] + M[3 * a + 2] * v[2];
}
/* lab = Q^T local:  o_b = sum_a Q_ab v_a */
static void matT_vec(const double M[9], const double v[3], double o[3]) {
  for (int b = 0; b < 3; ++b) o[b] = M[0 + b] * v[0] + M[3 + b] * v[1] + M[6 + b] * v[2];
}
static void mat_mul(const double A[9], const double B[9], double C[9]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) C[3 * a + b] = A[3 * a + 0] * B[0 + b] + A[3 * a + 1] * B[3 + b] + A[3 * a + 2] * B[6 + b];
}
/* A B^T */
static void mat_mul_T(const double A[9], const double B[9], double C[9]) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) C[3 * a + b] = A[3 * a + 0] * B[3 * b + 0] + A[3 * a + 1] * B[3 * b + 1] + A[3 * a + 2] * B[3 * b + 2];
}

/* ---------------------------------------------------------------- per-rod constants */

typedef struct {
  double A, I[3], B[3], S[3], rho;
} rod_consts;

/* A = pi r^2, I1 = I2 = pi r^4/4, I3 = I1 + I2, B = diag(E I1, E I2, G I3),
 * S = diag(alpha G A, alpha G A, E A)   (Methods, definitions after the strain measures) */
static rod_consts consts_of(const orc_params* p, int r) {
  rod_consts c;
  double rad = p->radius[r];
  double E = p->youngs[r], G = p->shear_mod[r];
  c.A = M_PI * rad * rad;
  c.I[0] = M_PI * rad * rad * rad * rad / 4.0;
  c.I[1] = c.I[0];
  c.I[2] = c.I[0] + c.I[1];
  c.B[0] = E * c.I[0];
  c.B[1] = E * c.I[1];
  c.B[2] = G * c.I[2];
  c.S[0] = p->alpha_c * G * c.A;
  c.S[1] = p->alpha_c * G * c.A;
  c.S[2] = E * c.A;
  c.rho = p->density[r];
  return c;
}

/* ---------------------------------------------------------------- rotations */

/* R = exp([phi]x) = I + (sin th/th) K + ((1 - cos th)/th^2) K^2, th = |phi|, K = [phi]x.
 * (1 - cos th) is written as 2 sin^2(th/2) to avoid cancellation at small th. */
void orc_rot_exp(const double phi[3], double R[9]) {
  double th = sqrt(dot3(phi, phi));
  double a, b;
  if (th == 0.0) {
    a = 1.0;
    b = 0.5;
  } else {
    double sh = sin(0.5 * th) / th;
    a = sin(th) / th;
    b = 2.0 * sh * sh;
  }
  double K[9] = {0.0, -phi[2], phi[1], phi[2], 0.0, -phi[0], -phi[1], phi[0], 0.0};
  double K2[9];
  mat_mul(K, K, K2);
  for (int q = 0; q < 9; ++q) R[q] = a * K[q] + b * K2[q];
  R[0] += 1.0;
  R[4] += 1.0;
  R[8] += 1.0;
}

/* phi = ax(log R): w = ax((R - R^T)/2) = sin(th) u, cos th = (tr R - 1)/2,
 * th = atan2(|w|, cos th), phi = th w/|w|  (zero rotation when |w| = 0). */
void orc_rot_log(const double R[9], double phi[3]) {
  double w[3] = {0.5 * (R[7] - R[5]), 0.5 * (R[2] - R[6]), 0.5 * (R[3] - R[1])};
  double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  double s = sqrt(dot3(w, w));
  if (s == 0.0) {
    phi[0] = phi[1] = phi[2] = 0.0;
    return;
  }
  double th = atan2(s, c);
  for (int q = 0; q < 3; ++q) phi[q] = th / s * w[q];
}

/* ---------------------------------------------------------------- validation */

static int validate(const orc_params* p) {
  if (p->n_rods <= 0) return fail("n_rods must be positive");
  for (int r = 0; r < p->n_rods; ++r) {
    if (p->n_elem[r] < 1) return fail("every rod needs at least one element");
    if (!(p->radius[r] > 0) || !(p->youngs[r] > 0) || !(p->shear_mod[r] > 0) || !(p->density[r] > 0))
      return fail("radius, moduli and density must be positive");
  }
  int64_t E = orc_num_elems(p);
  for (int64_t i = 0; i < E; ++i)
    if (!(p->rest_len[i] > 0)) return fail("rest lengths must be positive");
  if (p->act_amp)
    for (int r = 0; r < p->n_rods; ++r)
      if (!(p->act_period[r] > 0)) return fail("actuation period must be positive");
  if (p->muscle_amp)
    for (int r = 0; r < p->n_rods; ++r)
      if (!(p->muscle_period[r] > 0) || !(p->muscle_wavelength[r] > 0))
        return fail("muscle period and wavelength must be positive");
  if ((p->contact_mu < 0) || (p->contact_mu > 0 && !(p->contact_vslip > 0)))
    return fail("friction needs mu >= 0 and a positive slip velocity");
  if (p->n_walls < 0 || (p->n_walls > 0 && (!p->wall_point || !p->wall_normal)))
    return fail("walls need points and normals");
  for (int k = 0; k < p->n_walls; ++k) {
    const double* nn = p->wall_normal + 3 * k;
    if (fabs(dot3(nn, nn) - 1.0) > 1e-12) return fail("wall normals must be unit vectors");
  }
  if (p->n_walls > 0 && ((p->wall_mu < 0) || (p->wall_mu > 0 && !(p->wall_vslip > 0))))
    return fail("wall friction needs mu >= 0 and a positive slip velocity");
  return 0;
}

/* Regularised Coulomb friction at a contact with normal force fn >= 0 along unit nrm and
 * relative velocity vrel: -mu fn v_t / max(|v_t|, v_slip), v_t = vrel - (vrel . nrm) nrm
 * (Coulomb above the slip velocity, viscous below it; no tangential spring, so no history). */
static void friction_force(double mu, double vslip, double fn, const double nrm[3], const double vrel[3],
                           double ft[3]) {
  double vn = dot3(vrel, nrm), vt[3];
  for (int c = 0; c < 3; ++c) vt[c] = vrel[c] - vn * nrm[c];
  double sp = sqrt(dot3(vt, vt));
  double den = sp > vslip ? sp : vslip;
  for (int c = 0; c < 3; ++c) ft[c] = (mu > 0.0 && fn > 0.0) ? -mu * fn * vt[c] / den : 0.0;
}

/* ---------------------------------------------------------------- a3-a5: strains */

int orc_strains(const orc_params* p, const double* x, const double* Q, double* sigma, double* kappa,
                double* dil, double* vdil) {
  if (validate(p)) return -1;
  int64_t N = orc_num_nodes(p), E = orc_num_elems(p), V = orc_num_voronoi(p);
  rod_range* G = rod_ranges(p);
  if (!G) return fail("out of host memory");
  for (int r = 0; r < p->n_rods; ++r) {
    rod_range g = G[r];
    for (int i = 0; i < g.n; ++i) {
      int64_t ie = g.elem0 + i;
      double xa[3], xb[3], l[3], M[9], Ql[3];
      ld3(x, N, g.node0 + i, xa);
      ld3(x, N, g.node0 + i + 1, xb);
      for (int c = 0; c < 3; ++c) l[c] = xb[c] - xa[c];
      double rl = p->rest_len[ie];
      double ell = sqrt(dot3(l, l));
      ldQ(Q, E, ie, M);
      mat_vec(M, l, Ql);
      double s[3] = {Ql[0] / rl, Ql[1] / rl, Ql[2] / rl - 1.0};
      if (sigma) st3(sigma, E, ie, s);
      if (dil) dil[ie] = ell / rl;
    }
    for (int k = 0; k < g.n - 1; ++k) {
      int64_t ie = g.elem0 + k, iv = g.vor0 + k;
      double Ma[9], Mb[9], R[9], phi[3];
      ldQ(Q, E, ie, Ma);
      ldQ(Q, E, ie + 1, Mb);
      mat_mul_T(Mb, Ma, R); /* Q_{k+1} Q_k^T */
      orc_rot_log(R, phi);
      double D = 0.5 * (p->rest_len[ie] + p->rest_len[ie + 1]);
      double kap[3] = {-phi[0] / D, -phi[1] / D, -phi[2] / D};
      if (kappa) st3(kappa, V, iv, kap);
      if (vdil) {
        double xa[3], xb[3], xc[3], la[3], lb[3];
        ld3(x, N, g.node0 + k, xa);
        ld3(x, N, g.node0 + k + 1, xb);
        ld3(x, N, g.node0 + k + 2, xc);
        for (int c = 0; c < 3; ++c) {
          la[c] = xb[c] - xa[c];
          lb[c] = xc[c] - xb[c];
        }
        vdil[iv] = (sqrt(dot3(la, la)) + sqrt(dot3(lb, lb))) / (p->rest_len[ie] + p->rest_len[ie + 1]);
      }
    }
  }
  free(G);
  return 0;
}

/* ---------------------------------------------------------------- a8-a9: contact */

/* Closest points of P(s) = p0 + s d1 and R(u) = q0 + u d2 over [0,1]^2.
 * Minimises |r + s d1 - u d2|^2, r = p0 - q0.  Stationarity gives
 *   a s - b u = -c,  b s - e u = -f   with a = d1.d1, b = d1.d2, c = d1.r, e = d2.d2, f = d2.r,
 * so the free minimiser has s = (b f - c e)/(a e - b^2); s is clamped to [0,1], then
 * u = (b s + f)/e; if u leaves [0,1] it is clamped and s is recomputed from u and clamped
 * again (the clamped method for segment-segment distance).  Parallel segments
 * (a e - b^2 == 0) take s = 0. */
void orc_segment_closest(const double p0[3], const double p1[3], const double q0[3], const double q1[3],
                         double* s_out, double* u_out) {
  double d1[3], d2[3], r[3];
  for (int c = 0; c < 3; ++c) {
    d1[c] = p1[c] - p0[c];
    d2[c] = q1[c] - q0[c];
    r[c] = p0[c] - q0[c];
  }
  double a = dot3(d1, d1), e = dot3(d2, d2), f = dot3(d2, r);
  double s, u;
  if (a <= 0.0 && e <= 0.0) {
    s = 0.0;
    u = 0.0;
  } else if (a <= 0.0) {
    s = 0.0;
    u = f / e;
    u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
  } else {
    double c = dot3(d1, r);
    if (e <= 0.0) {
      u = 0.0;
      s = -c / a;
      s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
    } else {
      double b = dot3(d1, d2);
      double den = a * e - b * b;
      if (den != 0.0) {
        s = (b * f - c * e) / den;
        s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
      } else {
        s = 0.0;
      }
      u = (b * s + f) / e;
      if (u < 0.0) {
        u = 0.0;
        s = -c / a;
        s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
      } else if (u > 1.0) {
        u = 1.0;
        s = (b - c) / a;
        s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
      }
    }
  }
  *s_out = s;
  *u_out = u;
}

typedef struct {
  int64_t E, N;
  int32_t* rod_of;   /* segment -> rod */
  int64_t* node_of;  /* segment -> first node */
} seg_map;

static int build_seg_map(const orc_params* p, seg_map* m) {
  m->E = orc_num_elems(p);
  m->N = orc_num_nodes(p);
  m->rod_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)m->E);
  m->node_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)m->E);
  if (!m->rod_of || !m->node_of) return fail("out of host memory");
  int64_t ie = 0, jn = 0;
  for (int r = 0; r < p->n_rods; ++r) {
    for (int i = 0; i < p->n_elem[r]; ++i) {
      m->rod_of[ie] = r;
      m->node_of[ie] = jn + i;
      ++ie;
    }
    jn += p->n_elem[r] + 1;
  }
  return 0;
}
static void free_seg_map(seg_map* m) {
  free(m->rod_of);
  free(m->node_of);
}

/* Evaluate the pair (a, b), a < b.  Returns 1 and the force on segment a (f, applied with
 * weights 1-s, s on its nodes; -f with 1-u, u on the nodes of b) when the overlap is positive. */
static int pair_force(const orc_params* p, const seg_map* m, const double* x, const double* v, int64_t a, int64_t b,
                      double* s_out, double* u_out, double f[3], double* delta_out) {
  double p0[3], p1[3], q0[3], q1[3];
  int64_t na = m->node_of[a], nb = m->node_of[b];
  ld3(x, m->N, na, p0);
  ld3(x, m->N, na + 1, p1);
  ld3(x, m->N, nb, q0);
  ld3(x, m->N, nb + 1, q1);
  double s, u;
  orc_segment_closest(p0, p1, q0, q1, &s, &u);
  double pa[3], pb[3], dv[3];
  for (int c = 0; c < 3; ++c) {
    pa[c] = p0[c] + s * (p1[c] - p0[c]);
    pb[c] = q0[c] + u * (q1[c] - q0[c]);
    dv[c] = pa[c] - pb[c];
  }
  double d = sqrt(dot3(dv, dv));
  double delta = p->radius[m->rod_of[a]] + p->radius[m->rod_of[b]] - d;
  *s_out = s;
  *u_out = u;
  *delta_out = delta;
  if (!(delta > 0.0) || d == 0.0) return 0;
  double nrm[3] = {dv[0] / d, dv[1] / d, dv[2] / d};
  double fmag = p->contact_k * delta;
  if (v) {
    double va0[3], va1[3], vb0[3], vb1[3], vrel[3];
    ld3(v, m->N, na, va0);
    ld3(v, m->N, na + 1, va1);
    ld3(v, m->N, nb, vb0);
    ld3(v, m->N, nb + 1, vb1);
    for (int c = 0; c < 3; ++c) vrel[c] = ((1.0 - s) * va0[c] + s * va1[c]) - ((1.0 - u) * vb0[c] + u * vb1[c]);
    fmag = fmag - p->contact_c * dot3(vrel, nrm);
    if (fmag < 0.0) fmag = 0.0;
    double ft[3];
    friction_force(p->contact_mu, p->contact_vslip, fmag, nrm, vrel, ft);
    for (int c = 0; c < 3; ++c) f[c] = fmag * nrm[c] + ft[c];
    return 1;
  }
  if (fmag < 0.0) fmag = 0.0;
  for (int c = 0; c < 3; ++c) f[c] = fmag * nrm[c];
  return 1;
}

/* Uniform cell list over segment midpoints (counting sort by cell).  Cell size h is at least
 * 2 max radius + max current segment length, so any contacting pair has midpoints within
 * h of each other and therefore lies in the same or an adjacent cell. */
typedef struct {
  double lo[3], h;
  int64_t dim[3];
  int64_t* start; /* ncell + 1 */
  int64_t* order; /* segments sorted by cell */
  int64_t* cell_of;
} cell_list;

static int build_cell_list(const orc_params* p, const seg_map* m, const double* x, cell_list* cl) {
  int64_t E = m->E;
  double hmin = 0.0, rmax = 0.0, lmax = 0.0;
  for (int r = 0; r < p->n_rods; ++r)
    if (p->radius[r] > rmax) rmax = p->radius[r];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double* mid = (double*)malloc(sizeof(double) * 3 * (size_t)E);
  if (!mid) return fail("out of host memory");
  for (int64_t a = 0; a < E; ++a) {
    double p0[3], p1[3], l[3];
    ld3(x, m->N, m->node_of[a], p0);
    ld3(x, m->N, m->node_of[a] + 1, p1);
    for (int c = 0; c < 3; ++c) {
      l[c] = p1[c] - p0[c];
      mid[3 * a + c] = 0.5 * (p0[c] + p1[c]);
      if (mid[3 * a + c] < lo[c]) lo[c] = mid[3 * a + c];
      if (mid[3 * a + c] > hi[c]) hi[c] = mid[3 * a + c];
    }
    double ell = sqrt(dot3(l, l));
    if (ell > lmax) lmax = ell;
  }
  hmin = 2.0 * rmax + lmax;
  cl->h = p->cell_size > hmin ? p->cell_size : hmin;
  int64_t ncell = 1;
  for (int c = 0; c < 3; ++c) {
    if (!isfinite(lo[c]) || !isfinite(hi[c])) {
      free(mid);
      return fail("non-finite positions in contact broad phase");
    }
    cl->lo[c] = lo[c];
    cl->dim[c] = (int64_t)floor((hi[c] - lo[c]) / cl->h) + 1;
    ncell *= cl->dim[c];
  }
  if (ncell > ((int64_t)1 << 31)) {
    free(mid);
    return fail("cell grid too large");
  }
  cl->start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
  cl->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)E);
  cl->cell_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)E);
  if (!cl->start || !cl->order || !cl->cell_of) {
    free(mid);
    return fail("out of host memory");
  }
  for (int64_t a = 0; a < E; ++a) {
    int64_t ic[3];
    for (int c = 0; c < 3; ++c) {
      ic[c] = (int64_t)floor((mid[3 * a + c] - cl->lo[c]) / cl->h);
      if (ic[c] < 0) ic[c] = 0;
      if (ic[c] >= cl->dim[c]) ic[c] = cl->dim[c] - 1;
    }
    cl->cell_of[a] = (ic[2] * cl->dim[1] + ic[1]) * cl->dim[0] + ic[0];
    cl->start[cl->cell_of[a] + 1] += 1;
  }
  for (int64_t q = 0; q < ncell; ++q) cl->start[q + 1] += cl->start[q];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
  if (!fill) {
    free(mid);
    return fail("out of host memory");
  }
  memcpy(fill, cl->start, sizeof(int64_t) * (size_t)ncell);
  for (int64_t a = 0; a < E; ++a) cl->order[fill[cl->cell_of[a]]++] = a;
  free(fill);
  free(mid);
  return 0;
}
static void free_cell_list(cell_list* cl) {
  free(cl->start);
  free(cl->order);
  free(cl->cell_of);
}

/* Visit every pair (a < b) of segments of different rods that the chosen broad phase
 * proposes.  visit() returns nonzero to stop. */
typedef int (*pair_visitor)(int64_t a, int64_t b, void* ctx);

static int for_each_candidate(const orc_params* p, const seg_map* m, const double* x, pair_visitor visit, void* ctx) {
  if (p->broad_phase == 0) {
    for (int64_t a = 0; a < m->E; ++a)
      for (int64_t b = a + 1; b < m->E; ++b)
        if (m->rod_of[a] != m->rod_of[b])
          if (visit(a, b, ctx)) return 1;
    return 0;
  }
  cell_list cl;
  if (build_cell_list(p, m, x, &cl)) return -1;
  int stop = 0;
  for (int64_t a = 0; a < m->E && !stop; ++a) {
    int64_t c = cl.cell_of[a];
    int64_t ix = c % cl.dim[0], iy = (c / cl.dim[0]) % cl.dim[1], iz = c / (cl.dim[0] * cl.dim[1]);
    for (int dz = -1; dz <= 1 && !stop; ++dz)
      for (int dy = -1; dy <= 1 && !stop; ++dy)
        for (int dx = -1; dx <= 1 && !stop; ++dx) {
          int64_t jx = ix + dx, jy = iy + dy, jz = iz + dz;
          if (jx < 0 || jy < 0 || jz < 0 || jx >= cl.dim[0] || jy >= cl.dim[1] || jz >= cl.dim[2]) continue;
          int64_t cc = (jz * cl.dim[1] + jy) * cl.dim[0] + jx;
          for (int64_t q = cl.start[cc]; q < cl.start[cc + 1]; ++q) {
            int64_t b = cl.order[q];
            if (b > a && m->rod_of[a] != m->rod_of[b])
              if (visit(a, b, ctx)) {
                stop = 1;
                break;
              }
          }
        }
  }
  free_cell_list(&cl);
  return stop;
}

typedef struct {
  const orc_params* p;
  const seg_map* m;
  const double* x;
  const double* v;
  double* f;
  int64_t* pairs;
  int64_t cap, count;
} contact_ctx;

static int visit_force(int64_t a, int64_t b, void* vctx) {
  contact_ctx* C = (contact_ctx*)vctx;
  double s, u, f[3], delta;
  if (!pair_force(C->p, C->m, C->x, C->v, a, b, &s, &u, f, &delta)) return 0;
  int64_t na = C->m->node_of[a], nb = C->m->node_of[b], N = C->m->N;
  double wa = 1.0 - s;
  acc3(C->f, N, na, f, wa);
  acc3(C->f, N, na + 1, f, 1.0 - wa);
  acc3(C->f, N, nb, f, -(1.0 - u));
  acc3(C->f, N, nb + 1, f, -u);
  return 0;
}

static int visit_pair(int64_t a, int64_t b, void* vctx) {
  contact_ctx* C = (contact_ctx*)vctx;
  double s, u, f[3], delta;
  pair_force(C->p, C->m, C->x, NULL, a, b, &s, &u, f, &delta);
  if (delta > 0.0) {
    if (C->count < C->cap) {
      C->pairs[2 * C->count] = a;
      C->pairs[2 * C->count + 1] = b;
    }
    C->count++;
  }
  return 0;
}

int orc_contact_forces(const orc_params* p, const double* x, double* f, const double* v) {
  if (validate(p)) return -1;
  int64_t N = orc_num_nodes(p);
  memset(f, 0, sizeof(double) * 3 * (size_t)N);
  if (!p->contact) return 0;
  seg_map m;
  if (build_seg_map(p, &m)) return -1;
  contact_ctx C = {p, &m, x, v, f, NULL, 0, 0};
  int rc = for_each_candidate(p, &m, x, visit_force, &C);
  free_seg_map(&m);
  return rc < 0 ? -1 : 0;
}

int64_t orc_contact_pairs(const orc_params* p, const double* x, int64_t* pairs, int64_t cap) {
  if (validate(p)) return -1;
  seg_map m;
  if (build_seg_map(p, &m)) return -1;
  contact_ctx C = {p, &m, x, NULL, NULL, pairs, cap, 0};
  int rc = for_each_candidate(p, &m, x, visit_pair, &C);
  free_seg_map(&m);
  return rc < 0 ? -1 : C.count;
}

/* ---------------------------------------------------------------- a3-a7, a10: right-hand side */

static int act_element(const orc_params* p, int r) {
  int clamped = p->clamp_base && p->clamp_base[r];
  return (clamped && p->n_elem[r] >= 2) ? 1 : 0;
}

int orc_rhs(const orc_params* p, double t, const double* x, const double* v, const double* Q, const double* w,
            double* acc_v, double* acc_w) {
  if (validate(p)) return -1;
  int64_t N = orc_num_nodes(p), E = orc_num_elems(p), V = orc_num_voronoi(p);
  double* Nf = (double*)calloc(3 * (size_t)E, sizeof(double));  /* lab internal force per element */
  double* tau = (double*)calloc(3 * (size_t)E, sizeof(double)); /* local torque per element */
  double* dil = (double*)calloc((size_t)E, sizeof(double));
  double* P = (double*)calloc(3 * (size_t)(V > 0 ? V : 1), sizeof(double));
  double* T = (double*)calloc(3 * (size_t)(V > 0 ? V : 1), sizeof(double));
  double* ell = (double*)calloc((size_t)E, sizeof(double));
  double* fc = (double*)calloc(3 * (size_t)N, sizeof(double));
  rod_range* G = rod_ranges(p);
  int rc = 0;
  if (!Nf || !tau || !dil || !ell || !P || !T || !fc || !G) rc = fail("out of host memory");
  if (!rc && p->contact && orc_contact_forces(p, x, fc, v)) rc = -1;
  if (rc) goto done;

  /* rods are independent here (each writes only its own entries): the OpenMP build runs them
   * on all host cores, the plain build ignores the pragma */
#pragma omp parallel for schedule(dynamic, 8)
  for (int r = 0; r < p->n_rods; ++r) {
    rod_range g = G[r];
    rod_consts K = consts_of(p, r);
    /* elements: strain, internal force, shear couple, transport couples */
    for (int i = 0; i < g.n; ++i) {
      int64_t ie = g.elem0 + i;
      double xa[3], xb[3], va[3], vb[3], l[3], M[9], Ql[3], sig[3], nl[3], Nl[3], wi[3];
      ld3(x, N, g.node0 + i, xa);
      ld3(x, N, g.node0 + i + 1, xb);
      ld3(v, N, g.node0 + i, va);
      ld3(v, N, g.node0 + i + 1, vb);
      ld3(w, E, ie, wi);
      ldQ(Q, E, ie, M);
      double rl = p->rest_len[ie];
      for (int c = 0; c < 3; ++c) l[c] = xb[c] - xa[c];
      double lg = sqrt(dot3(l, l));
      double e = lg / rl;
      double tt[3] = {l[0] / lg, l[1] / lg, l[2] / lg};
      mat_vec(M, l, Ql);
      sig[0] = Ql[0] / rl;
      sig[1] = Ql[1] / rl;
      sig[2] = Ql[2] / rl - 1.0;
      if (p->rest_sigma)
        for (int c = 0; c < 3; ++c) sig[c] -= p->rest_sigma[c * E + ie];
      for (int c = 0; c < 3; ++c) nl[c] = K.S[c] * sig[c];
      matT_vec(M, nl, Nl);
      for (int c = 0; c < 3; ++c) Nl[c] = Nl[c] / e;
      st3(Nf, E, ie, Nl);
      dil[ie] = e;
      ell[ie] = lg;
      /* shear couple ((Q t) x n) rl */
      double Qt[3], ts[3];
      mat_vec(M, tt, Qt);
      cross3(Qt, nl, ts);
      /* transport couples (J w / e) x w + (J w / e^2) de/dt */
      double Jw[3], Jwe[3], tl[3];
      for (int c = 0; c < 3; ++c) Jw[c] = K.rho * rl * K.I[c] * wi[c];
      for (int c = 0; c < 3; ++c) Jwe[c] = Jw[c] / e;
      cross3(Jwe, wi, tl);
      double dv[3] = {vb[0] - va[0], vb[1] - va[1], vb[2] - va[2]};
      double edot = dot3(tt, dv) / rl;
      for (int c = 0; c < 3; ++c) tau[c * E + ie] = ts[c] * rl + tl[c] + Jw[c] / (e * e) * edot;
    }
    /* Voronoi points: curvature, bending moment, dilatation */
    for (int k = 0; k < g.n - 1; ++k) {
      int64_t ie = g.elem0 + k, iv = g.vor0 + k;
      double Ma[9], Mb[9], R[9], phi[3], kap[3], mk[3], kxm[3];
      ldQ(Q, E, ie, Ma);
      ldQ(Q, E, ie + 1, Mb);
      mat_mul_T(Mb, Ma, R);
      orc_rot_log(R, phi);
      double rla = p->rest_len[ie], rlb = p->rest_len[ie + 1];
      double D = 0.5 * (rla + rlb);
      for (int c = 0; c < 3; ++c) kap[c] = -phi[c] / D;
      double eps = (ell[ie] + ell[ie + 1]) / (rla + rlb);
      double eps3 = eps * eps * eps;
      for (int c = 0; c < 3; ++c) {
        double k0 = p->rest_kappa ? p->rest_kappa[c * V + iv] : 0.0;
        mk[c] = K.B[c] * (kap[c] - k0);
      }
      cross3(kap, mk, kxm);
      for (int c = 0; c < 3; ++c) {
        P[c * V + iv] = mk[c] / eps3;
        T[c * V + iv] = kxm[c] * D / eps3;
      }
    }
    /* element angular accelerations */
    int iact = act_element(p, r);
    double bt[3] = {0.0, 0.0, 0.0};
    if (p->magnetization)
      for (int c = 0; c < 3; ++c)
        bt[c] = p->field_b0[c] + p->field_bc[c] * cos(p->field_omega * t) + p->field_bs[c] * sin(p->field_omega * t);
    for (int i = 0; i < g.n; ++i) {
      int64_t ie = g.elem0 + i;
      double tot[3], wi[3];
      ld3(w, E, ie, wi);
      double rl = p->rest_len[ie];
      for (int c = 0; c < 3; ++c) {
        double Pi = (i <= g.n - 2) ? P[c * V + g.vor0 + i] : 0.0;
        double Pm = (i >= 1) ? P[c * V + g.vor0 + i - 1] : 0.0;
        double Ti = (i <= g.n - 2) ? T[c * V + g.vor0 + i] : 0.0;
        double Tm = (i >= 1) ? T[c * V + g.vor0 + i - 1] : 0.0;
        tot[c] = (Pi - Pm) + 0.5 * (Tm + Ti) + tau[c * E + ie];
        tot[c] += -p->nu_damp * rl * (K.I[c] / K.A) * wi[c];
        if (p->elem_couple) tot[c] += p->elem_couple[c * E + ie];
      }
      if (p->act_amp && i == iact)
        tot[0] += p->act_amp[r] * sin(2.0 * M_PI * t / p->act_period[r] + p->act_phase[r]);
      if (p->magnetization) {
        /* rl (m x (Q b)) with Q b the field in the element's frame */
        double M[9], qb[3], mi[3], cmag[3];
        ldQ(Q, E, ie, M);
        for (int a = 0; a < 3; ++a)
          qb[a] = M[3 * a] * bt[0] + M[3 * a + 1] * bt[1] + M[3 * a + 2] * bt[2];
        ld3(p->magnetization, E, ie, mi);
        cross3(mi, qb, cmag);
        for (int c = 0; c < 3; ++c) tot[c] += rl * cmag[c];
      }
      if (p->muscle_amp && g.n >= 2) {
        /* tau_k at the Voronoi points on both sides of element i (k = i - 1 and k = i) */
        double s_right = 0.0;
        for (int q = 0; q <= i; ++q) s_right += p->rest_len[g.elem0 + q];   /* arc length of node i+1 */
        double s_left = s_right - rl;                                         /* arc length of node i */
        double om = 2.0 * M_PI / p->muscle_period[r], kw = 2.0 * M_PI / p->muscle_wavelength[r];
        double tr = (i <= g.n - 2) ? p->muscle_amp[r] * sin(om * t - kw * s_right + p->muscle_phase[r]) : 0.0;
        double tl = (i >= 1) ? p->muscle_amp[r] * sin(om * t - kw * s_left + p->muscle_phase[r]) : 0.0;
        tot[0] += tl - tr;
      }
      for (int c = 0; c < 3; ++c) acc_w[c * E + ie] = dil[ie] * tot[c] / (K.rho * rl * K.I[c]);
    }
    /* node accelerations */
    for (int j = 0; j <= g.n; ++j) {
      int64_t jn = g.node0 + j;
      double rl_l = (j >= 1) ? p->rest_len[g.elem0 + j - 1] : 0.0;
      double rl_r = (j <= g.n - 1) ? p->rest_len[g.elem0 + j] : 0.0;
      double mass = 0.5 * K.rho * K.A * (rl_l + rl_r);
      double rlN = 0.5 * (rl_l + rl_r);
      double F[3], vj[3];
      ld3(v, N, jn, vj);
      for (int c = 0; c < 3; ++c) {
        double Nr = (j <= g.n - 1) ? Nf[c * E + g.elem0 + j] : 0.0;
        double Nlft = (j >= 1) ? Nf[c * E + g.elem0 + j - 1] : 0.0;
        F[c] = Nr - Nlft;
        F[c] += mass * p->gravity[c];
        F[c] += -(p->nu_damp + p->stokes_gamma) * rlN * vj[c];
        F[c] += fc[c * N + jn];
        if (p->tip_force && j == g.n) F[c] += p->tip_force[c * p->n_rods + r];
      }
      for (int k = 0; k < p->n_walls; ++k) {
        /* node sphere of radius r against the half-space n . (x - p - u t) >= 0 */
        const double* nn = p->wall_normal + 3 * k;
        double xj[3], d[3], u[3] = {0.0, 0.0, 0.0}, vrel[3];
        ld3(x, N, jn, xj);
        if (p->wall_velocity)
          for (int c = 0; c < 3; ++c) u[c] = p->wall_velocity[3 * k + c];
        for (int c = 0; c < 3; ++c) d[c] = xj[c] - (p->wall_point[3 * k + c] + u[c] * t);
        double delta = p->radius[r] - dot3(d, nn);
        if (!(delta > 0.0)) continue;
        for (int c = 0; c < 3; ++c) vrel[c] = vj[c] - u[c];
        double fn = p->wall_k * delta - p->wall_c * dot3(vrel, nn);
        if (fn < 0.0) fn = 0.0;
        double ft[3];
        friction_force(p->wall_mu, p->wall_vslip, fn, nn, vrel, ft);
        for (int c = 0; c < 3; ++c) F[c] += fn * nn[c] + ft[c];
      }
      for (int c = 0; c < 3; ++c) acc_v[c * N + jn] = F[c] / mass;
    }
    /* constraint on rates */
    if (p->clamp_base && p->clamp_base[r]) {
      for (int c = 0; c < 3; ++c) {
        acc_v[c * N + g.node0] = 0.0;
        acc_w[c * E + g.elem0] = 0.0;
      }
    }
  }
done:
  free(Nf);
  free(tau);
  free(dil);
  free(ell);
  free(P);
  free(T);
  free(fc);
  free(G);
  return rc;
}

/* ---------------------------------------------------------------- a1/a11, a2, a10, a12: stepping */

static void kinematic_half(const orc_params* p, double h, double* x, const double* v, double* Q, const double* w) {
  int64_t N = orc_num_nodes(p), E = orc_num_elems(p);
#pragma omp parallel for
  for (int64_t j = 0; j < N; ++j)
    for (int c = 0; c < 3; ++c) x[c * N + j] += h * v[c * N + j];
#pragma omp parallel for
  for (int64_t i = 0; i < E; ++i) {
    double M[9], R[9], Mn[9], phi[3];
    for (int c = 0; c < 3; ++c) phi[c] = -h * w[c * E + i];
    orc_rot_exp(phi, R);
    ldQ(Q, E, i, M);
    mat_mul(R, M, Mn);
    stQ(Q, E, i, Mn);
  }
}

typedef struct {
  double x0[3], Q0[9];
} clamp_value;

static void constrain_values(const orc_params* p, const rod_range* G, const clamp_value* cv, double* x, double* Q) {
  if (!p->clamp_base) return;
  int64_t N = orc_num_nodes(p), E = orc_num_elems(p);
  for (int r = 0; r < p->n_rods; ++r) {
    if (!p->clamp_base[r]) continue;
    rod_range g = G[r];
    st3(x, N, g.node0, cv[r].x0);
    stQ(Q, E, g.elem0, cv[r].Q0);
  }
}
static void constrain_rates(const orc_params* p, const rod_range* G, double* v, double* w) {
  if (!p->clamp_base) return;
  int64_t N = orc_num_nodes(p), E = orc_num_elems(p);
  for (int r = 0; r < p->n_rods; ++r) {
    if (!p->clamp_base[r]) continue;
    rod_range g = G[r];
    for (int c = 0; c < 3; ++c) {
      v[c * N + g.node0] = 0.0;
      w[c * E + g.elem0] = 0.0;
    }
  }
}

int orc_step(const orc_params* p, double t, double dt, int64_t n_steps, double* x, double* v, double* Q, double* w) {
  if (validate(p)) return -1;
  int64_t N = orc_num_nodes(p), E = orc_num_elems(p);
  double* av = (double*)malloc(sizeof(double) * 3 * (size_t)N);
  double* aw = (double*)malloc(sizeof(double) * 3 * (size_t)E);
  clamp_value* cv = (clamp_value*)malloc(sizeof(clamp_value) * (size_t)p->n_rods);
  rod_range* G = rod_ranges(p);
  if (!av || !aw || !cv || !G) return fail("out of host memory");
  for (int r = 0; r < p->n_rods; ++r) {
    rod_range g = G[r];
    ld3(x, N, g.node0, cv[r].x0);
    ldQ(Q, E, g.elem0, cv[r].Q0);
  }
  int rc = 0;
  for (int64_t s = 0; s < n_steps; ++s) {
    kinematic_half(p, 0.5 * dt, x, v, Q, w);
    constrain_values(p, G, cv, x, Q);
    if (orc_rhs(p, t + 0.5 * dt, x, v, Q, w, av, aw)) {
      rc = -1;
      break;
    }
#pragma omp parallel for
    for (int64_t q = 0; q < 3 * N; ++q) v[q] += dt * av[q];
#pragma omp parallel for
    for (int64_t q = 0; q < 3 * E; ++q) w[q] += dt * aw[q];
    constrain_rates(p, G, v, w);
    kinematic_half(p, 0.5 * dt, x, v, Q, w);
    constrain_values(p, G, cv, x, Q);
    t += dt;
  }
  free(av);
  free(aw);
  free(cv);
  free(G);
  return rc;
}

/* ---------------------------------------------------------------- diagnostics */

double orc_energy(const orc_params* p, const double* x, const double* v, const double* Q, const double* w) {
  if (validate(p)) return NAN;
  int64_t N = orc_num_nodes(p), E = orc_num_elems(p), V = orc_num_voronoi(p);
  double* sig = (double*)malloc(sizeof(double) * 3 * (size_t)E);
  double* kap = (double*)malloc(sizeof(double) * 3 * (size_t)(V > 0 ? V : 1));
  if (!sig || !kap) return NAN;
  orc_strains(p, x, Q, sig, kap, NULL, NULL);
  rod_range* G = rod_ranges(p);
  if (!G) return NAN;
  double H = 0.0;
  for (int r = 0; r < p->n_rods; ++r) {
    rod_range g = G[r];
    rod_consts K = consts_of(p, r);
    for (int j = 0; j <= g.n; ++j) {
      int64_t jn = g.node0 + j;
      double rl_l = (j >= 1) ? p->rest_len[g.elem0 + j - 1] : 0.0;
      double rl_r = (j <= g.n - 1) ? p->rest_len[g.elem0 + j] : 0.0;
      double mass = 0.5 * K.rho * K.A * (rl_l + rl_r);
      double vj[3], xj[3];
      ld3(v, N, jn, vj);
      ld3(x, N, jn, xj);
      H += 0.5 * mass * dot3(vj, vj);
      H -= mass * dot3(p->gravity, xj);
      if (p->tip_force && j == g.n) {
        double F[3] = {p->tip_force[r], p->tip_force[p->n_rods + r], p->tip_force[2 * p->n_rods + r]};
        H -= dot3(F, xj);
      }
    }
    for (int i = 0; i < g.n; ++i) {
      int64_t ie = g.elem0 + i;
      double rl = p->rest_len[ie];
      for (int c = 0; c < 3; ++c) {
        double wc = w[c * E + ie];
        double sc = sig[c * E + ie] - (p->rest_sigma ? p->rest_sigma[c * E + ie] : 0.0);
        H += 0.5 * K.rho * rl * K.I[c] * wc * wc;
        H += 0.5 * rl * K.S[c] * sc * sc;
      }
    }
    for (int k = 0; k < g.n - 1; ++k) {
      int64_t iv = g.vor0 + k;
      double D = 0.5 * (p->rest_len[g.elem0 + k] + p->rest_len[g.elem0 + k + 1]);
      for (int c = 0; c < 3; ++c) {
        double kc = kap[c * V + iv] - (p->rest_kappa ? p->rest_kappa[c * V + iv] : 0.0);
        H += 0.5 * D * K.B[c] * kc * kc;
      }
    }
  }
  free(sig);
  free(kap);
  free(G);
  return H;
}

double orc_orthonormality_error(const orc_params* p, const double* Q) {
  int64_t E = orc_num_elems(p);
  double worst = 0.0;
  for (int64_t i = 0; i < E; ++i) {
    double M[9], P[9];
    ldQ(Q, E, i, M);
    mat_mul_T(M, M, P);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double d = fabs(P[3 * a + b] - (a == b ? 1.0 : 0.0));
        if (d > worst) worst = d;
      }
  }
  return worst;
}
