// rod_internal.h -- structures shared by the translation units of librod (host + device).
// Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rod {

// Device error word bits (latched; the host maps them to rod_status).
enum : int {
  ERR_NONFINITE = 1,
  ERR_OVERFLOW = 2,
  ERR_TIMEOUT = 4,    // a bounded wait of the surrogate's fused kernel ran out
  ERR_GRID = 8,       // a segment longer than the contact cell allows
};

// Per-rod constants, derived once at create time from the description (Methods: A = pi r^2,
// I1 = I2 = pi r^4/4, I3 = I1 + I2, B = diag(E I1, E I2, G I3), S = diag(aG A, aG A, E A)).
struct RodConst {
  double S[3];          // shear/stretch stiffness
  double B[3];          // bend/twist stiffness
  double rhoI[3];       // rho I_c (element inertia is rhoI * rest length)
  double inv_rhoI[3];   // 1 / (rho I_c)
  double damp_lin;      // (nu + gamma) / (rho A): translational decay rate
  double damp_rot;      // nu / (rho A): rotational decay rate
  double act_amp;       // base couple amplitude (0: none)
  double act_omega;     // 2 pi / T
  double act_phase;
  double tip[3];        // tip force (lab)
  double radius;
  int32_t node0;        // first node (global)
  int32_t elem0;        // first element (global)
  int32_t n;            // elements
  int32_t clamp;        // 1: node 0 + element 0 held
  int32_t act_elem;     // rod-local element carrying the base couple (-1: none)
  float radius_f;       // radius rounded to FP32 (contact culling)
  double muscle_amp;    // travelling-wave muscle couple amplitude (0: none)
  double muscle_omega;  // 2 pi / T
  double muscle_k;      // 2 pi / lambda
  double muscle_phase;
  // circular cross-section: I1 = I2, so S[0] = S[1], B[0] = B[1], rhoI[0] = rhoI[1]; the step
  // folds the products that these equalities make redundant, with
  double rhoI_12;       // rhoI[1] - rhoI[2]: (rho I w) x w = rhoI_12 (w1 w2, -w0 w2, 0)
  double B_21;          // B[2] - B[1]: kappa x (B kappa) = B_21 (k1 k2, -k0 k2, 0)
  double B_21q;         // B_21 / 4 (the factor D / (2 D) = 1/2 of the Voronoi couple, times the
                        // trapezoid's 1/2)
};

constexpr int kMaxWalls = 8;

// A thread block's share of the ensemble: consecutive rods (listed = 0: rod0.. and the global
// first element, node and Voronoi point), or any rods (listed = 1: entries list_off ..
// list_off + nrods of StepParams::pack_rods), with the pack's element, node and Voronoi counts.
struct Pack {
  int32_t rod0, nrods;
  int32_t elem0, nelem;  // global first element (consecutive packs), element count
  int32_t node0, nnode;  // global first node (consecutive packs), node count
  int32_t vor0, nvor;    // global first Voronoi point (consecutive packs), count
  int32_t listed, list_off;
};

// Read-only parameters of the step kernels.
// Arguments of the contact kernels (device pointers of the contact state and its parameters).
struct ContactArgs {
  const double* x;
  const double* v;
  const int* seg_rod;
  const int* seg_cell;
  const int* cell_start;
  const int* sorted;
  const float4* prox;
  const float4* recA;
  const int4* recB;
  const float4* recC;
  const int* gate;
  int* nbr;
  int* nbr_count;
  const int* slot_of;
  const float4* seg_prox;
  unsigned* active_mask;
  int* active;
  int* n_active;
  float skin;
  const RodConst* rods;
  double* fseg;
  int* err;
  int64_t N, E;
  int dim[3];
  double k, c;
  double mu, vslip, inv_vslip;
};

struct StepParams {
  // state (component-major)
  double* x;
  double* v;
  double* Q;
  double* w;
  int64_t N, E, V;
  // per-item constants
  const double* rest_len;     // [E]
  const double* inv_rl;       // [E]  1/rl
  const double* inv_2D;       // [V]  1/(rl_k + rl_{k+1}) = 1/(2 D_k)
  const double* sq_2D;        // [V]  (rl_k + rl_{k+1})^2 = (2 D_k)^2
  const double* Dhat;         // [V]  D_k
  const double* inv_rl2;      // [E]  1/rl^2
  const double* inv_m;        // [N]  1/lumped mass
  const double* rest_kappa;   // [3V] or null
  const double* rest_sigma;   // [3E] or null
  const double* elem_couple;  // [3E] or null
  const double* clamp_x;      // [3R] values held by the clamp
  const double* clamp_Q;      // [9R]
  const RodConst* rods;       // [R]
  const Pack* packs;
  const int2* pack_rods;      // listed packs: (global rod, first pack-local element) per entry
  int32_t n_packs;
  int32_t n_rods;
  double gravity[3];
  int32_t has_gravity;
  int32_t has_damp_lin;       // some rod has linear damping or drag (damp_lin != 0)
  int32_t has_damp_rot;       // some rod has rotational damping (damp_rot != 0)
  int32_t has_tip;            // some rod has a tip force
  int32_t has_act;
  // magnetic couple rl (m x (Q b(t))): m per unit reference length (local) [3E] or null
  const double* magnet;
  double field_b0[3], field_bc[3], field_bs[3], field_omega;
  // travelling-wave muscle couples: rest arc length of each element's first node [E] (null: none)
  const double* arc0;
  // walls
  int32_t n_walls;
  double wall_p[kMaxWalls][3], wall_n[kMaxWalls][3], wall_u[kMaxWalls][3];
  double wall_k, wall_c, wall_mu, wall_vslip;
  // contact: per-segment node forces [6E] (force on node a = first node, node b), or null
  const double* fseg;
  // skin-list contact: bit e set when segment e has candidates (its fseg entries are written);
  // null: every segment's entries are written
  const unsigned* fmask;
  int* err;                   // device error word
  // simulated time of the state at launch (device scalar; replayed graphs read it), or null
  const double* t_dev;
  // contact binning of the positions a half/one-step launch leaves behind, or bin_count = null
  float4* bin_prox;           // [E] FP32 midpoint + half length
  int* bin_cell;              // [E]
  int* bin_count;             // [cells] counts (zeroed by the caller)
  float bin_lo[3];
  float bin_inv_h;
  int bin_dim[3];
  float bin_l_allowed;        // longest element the cell covers, less the FP32 rounding margin
  // skin-list contact: an upper bound of the largest squared node displacement since the list
  // was built, raised by every launch with the bits of a non-negative double (disp_ref = null:
  // not tracked), and the FP32 segment proxies of the positions a half/one-step launch leaves
  // behind: [2e] = (midpoint, half length), [2e + 1] = (half edge, radius); null: not written
  const float* disp_ref;      // [3N] positions of the last list build, rounded to FP32
  unsigned long long* disp_word;
  float4* seg_prox;           // [2E]
  // byte offset of the FP32 node positions in a block's dynamic shared memory (0: none; set by
  // the launcher when the proxies are written and the shape leaves room for them)
  int32_t xf_smem_off;
  // host side only: packs of rods too long for a block (one rod each) and the global scratch
  // their cooperative launches use as working memory
  const struct Pack* long_packs_h;
  int32_t n_long;
  double* long_scratch;
};

// Kernel classes for the optional per-kernel timing (rod_system_profile).
enum KernelClass : int {
  K_PACK_STEPS = 0, K_PACK_ONE_STEP, K_KIN_HALF, K_RHS, K_CONTACT_BIN, K_CONTACT_SCAN, K_CONTACT_SCATTER,
  K_CONTACT_SORT, K_CONTACT_GATHER, K_CONTACT_NODE_FORCES, K_CONTACT_LIST_BUILD, K_CONTACT_LIST_FORCE, K_MISC,
  K_NUM_CLASSES
};
const char* kernel_class_name(int k);

// Called around every kernel launch: counts launches and, when profiling, records CUDA events
// on the launching stream.
struct LaunchHook {
  void (*fn)(void* ctx, int cls, int phase, cudaStream_t st) = nullptr;  // phase 0 = before, 1 = after
  void* ctx = nullptr;
  void before(int cls, cudaStream_t st) const { if (fn) fn(ctx, cls, 0, st); }
  void after(int cls, cudaStream_t st) const { if (fn) fn(ctx, cls, 1, st); }
};

// Launch shape of the pack kernels.
struct LaunchShape {
  int32_t cap_elems;   // elements per block (pack capacity)
  int32_t cap_rods;    // rods per block
  int32_t threads;
};

size_t step_smem_bytes(const LaunchShape& s);
// Largest dynamic shared memory of one block (opt-in) on this part.
constexpr size_t kMaxBlockSmem = 227 * 1024;

// Kernel launchers (rod_step.cu).
enum StepMode : int { MODE_STEPS = 0, MODE_RHS = 1, MODE_KIN_HALF = 2, MODE_ONE_STEP = 3 };
cudaError_t launch_pack_kernel(const StepParams& P, const LaunchShape& s, int mode, int64_t n_steps, double t0,
                               double dt, int last_half, double* acc_v, double* acc_w, cudaStream_t st,
                               const LaunchHook& hook);

}  // namespace rod
