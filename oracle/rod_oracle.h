/*
 * rod_oracle.h -- plain, slow, FP64 CPU oracle for the discrete Cosserat-rod step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * code: only the tests, the package's smoke check and the benchmark's CPU-baseline leg do.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes follows the paper's statement of the model:
 *   - Cosserat rod kinematics, strains sigma = Q(r' - d3), curvature kappa = ax(Q dQ^T/ds),
 *     angular velocity omega = ax(Q dQ^T/dt), B, S, I tensors (Methods, "Cosserat rod dynamics");
 *   - linear and angular momentum balance (Methods, Eq. 1a and Eq. 1b);
 *   - multi-stage symplectic (Verlet) time integration with kinematic constraints enforced
 *     after every stage (Results, "Performance-oriented software design");
 *   - rod-rod contact by a normal spring-dashpot force (Results, "Fibrous granular materials"),
 *     with an exhaustive O(N^2) broad phase and a uniform-grid broad phase (same section, Fig. 2e),
 *     and inter-filament friction (same section);
 *   - the magnetic couple of magnetized filaments (Methods, Eq. 2), travelling-wave muscle
 *     couples (Results, active filaments) and rod-wall contact (rod-boundary contact, Results).
 * The discrete scheme (staggered nodes/elements/Voronoi points, difference and averaging
 * operators with zero ghosts, lumped masses) is the standard one of the method paper the
 * authors cite for the discretisation; every place where the paper is silent is a documented
 * reading (listed in the repository's design notes and in rod_oracle.c).
 *
 * Layout (shared with the tests, not with the CUDA code): rods packed one after another
 * (CSR order).  Rod r has n_r elements, n_r+1 nodes, n_r-1 Voronoi points.
 * Every per-item vector is stored component-major ("SoA"): x[c*N + j], c = 0,1,2.
 * Directors: Q[(3a+b)*E + i] = b-th lab component of director d_{a+1} of element i
 * (the rows of the director matrix Q are d1, d2, d3).
 */
#ifndef ROD_ORACLE_H
#define ROD_ORACLE_H
#include <stdint.h>

/* ORC_CXX_LINKAGE: the C++ builds of this source over other number types (oracle_ad.cpp)
 * give the functions C++ linkage inside a namespace of their own. */
#if defined(__cplusplus) && !defined(ORC_CXX_LINKAGE)
extern "C" {
#endif

typedef struct {
  int32_t n_rods;
  const int32_t* n_elem;        /* n_rods */
  const double* rest_len;       /* E: element rest lengths */
  const double* radius;         /* n_rods */
  const double* youngs;         /* n_rods, E */
  const double* shear_mod;      /* n_rods, G */
  const double* density;        /* n_rods, volumetric rho */
  double alpha_c;               /* shear correction coefficient */
  const int8_t* clamp_base;     /* n_rods or NULL: node 0 and element 0 held at their initial values */
  const double* rest_kappa;     /* 3*V or NULL */
  const double* rest_sigma;     /* 3*E or NULL */
  double gravity[3];
  double nu_damp;               /* linear damping: force -nu v per length, couple -nu (I/A) w per length */
  double stokes_gamma;          /* isotropic drag per unit length (force only) */
  const double* tip_force;      /* 3*n_rods (component-major) or NULL, applied at the last node */
  const double* act_amp;        /* n_rods or NULL: base couple amplitude about local d1 */
  const double* act_period;     /* n_rods */
  const double* act_phase;      /* n_rods */
  const double* elem_couple;    /* 3*E or NULL: constant local couples per element */
  /* contact */
  int32_t contact;              /* 0 = off, 1 = on */
  double contact_k, contact_c;  /* spring stiffness, dashpot coefficient */
  double cell_size;             /* <= 0: 2*max radius + current max element length */
  int32_t broad_phase;          /* 0 = exhaustive O(N^2), 1 = uniform cell list */
  /* magnetic couple (Methods, "Magnetized filaments", Eq. 2): c = m x (Q b(t)) per unit
   * reference length, element couple rl c; b(t) = b0 + bc cos(omega t) + bs sin(omega t) (lab) */
  const double* magnetization;  /* 3*E or NULL: m per unit reference length, local frame */
  double field_b0[3], field_bc[3], field_bs[3];
  double field_omega;
  /* travelling-wave muscle couples (the self-activation of the active-filament study): at
   * interior Voronoi point k of rod r, tau_k = A sin(2 pi t / T - 2 pi s_k / lambda + phi)
   * about local d1, s_k the rest arc length of that point; element i receives
   * tau_{i-1} - tau_i (zero outside the rod), so the couples sum to zero along the rod */
  const double* muscle_amp;        /* n_rods or NULL */
  const double* muscle_period;     /* n_rods, T > 0 */
  const double* muscle_wavelength; /* n_rods, lambda > 0 */
  const double* muscle_phase;      /* n_rods */
  /* rod-rod friction: regularised Coulomb force -mu f_n v_t / max(|v_t|, v_slip) at the
   * closest points (v_t: tangential part of the relative velocity), split like the normal force */
  double contact_mu, contact_vslip;
  /* walls: half-spaces n . (x - p - u t) >= r of the node spheres (radius r of the rod);
   * normal force max(0, k delta - c v_rel . n) n, friction as above with the wall's mu, v_slip */
  int32_t n_walls;
  const double* wall_point;     /* [n_walls][3] */
  const double* wall_normal;    /* [n_walls][3], unit */
  const double* wall_velocity;  /* [n_walls][3] or NULL */
  double wall_k, wall_c, wall_mu, wall_vslip;
} orc_params;

/* sizes */
int64_t orc_num_nodes(const orc_params* p);
int64_t orc_num_elems(const orc_params* p);
int64_t orc_num_voronoi(const orc_params* p);

/* rotations (Methods: Q proper orthogonal, ax operator) */
void orc_rot_exp(const double phi[3], double R[9]);      /* R = exp([phi]x), row-major */
void orc_rot_log(const double R[9], double phi[3]);      /* phi = ax(log R) */

/* strains and curvature of the current configuration (a3-a5) */
int orc_strains(const orc_params* p, const double* x, const double* Q,
                double* sigma /*3E*/, double* kappa /*3V*/, double* dil /*E*/, double* vdil /*V*/);

/* contact forces on nodes at positions x, velocities v (a8-a9); f is overwritten (3N) */
int orc_contact_forces(const orc_params* p, const double* x, double* f, const double* v);

/* contact pairs with positive overlap: writes up to cap pairs (seg_i < seg_j), returns count or <0 */
int64_t orc_contact_pairs(const orc_params* p, const double* x, int64_t* pairs, int64_t cap);

/* closest points of segments P(s)=p0+s(p1-p0), R(u)=q0+u(q1-q0) on [0,1]^2 */
void orc_segment_closest(const double p0[3], const double p1[3], const double q0[3], const double q1[3],
                         double* s, double* u);

/* right-hand side (a3-a7 + a10 without the update): accelerations of nodes (3N) and
 * angular accelerations of elements (3E) at time t; contact forces included when enabled. */
int orc_rhs(const orc_params* p, double t, const double* x, const double* v, const double* Q,
            const double* w, double* acc_v, double* acc_w);

/* n_steps full position-Verlet steps from time t (a1-a12). State arrays updated in place. */
int orc_step(const orc_params* p, double t, double dt, int64_t n_steps,
             double* x, double* v, double* Q, double* w);

/* total energy: kinetic + elastic - work potential of gravity and tip force */
double orc_energy(const orc_params* p, const double* x, const double* v, const double* Q, const double* w);

/* max over elements of |Q Q^T - I|_inf */
double orc_orthonormality_error(const orc_params* p, const double* Q);

/* last error message */
const char* orc_last_error(void);

#if defined(__cplusplus) && !defined(ORC_CXX_LINKAGE)
}
#endif
#endif
