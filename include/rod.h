/*
 * rod.h -- C ABI of the GB300 (sm_103a) Cosserat-rod library (librod.so).
 *
 * One FP64 explicit time step over an ensemble of discrete Cosserat rods:
 *   strains sigma = Q(r' - d3) and curvature kappa = ax(Q dQ^T/ds) (Methods, "Cosserat rod
 *   dynamics"), linear and angular momentum balance (Methods, Eq. 1a, Eq. 1b), external,
 *   damping and drag loads (f, c of Eq. 1), rod-rod contact by a normal spring-dashpot over a
 *   uniform cell list (Results, "Fibrous granular materials", Fig. 2e), advanced by a
 *   multi-stage symplectic (position Verlet) scheme with kinematic constraints after every
 *   stage and an exponential-map director update (Results, "Performance-oriented software
 *   design").
 *
 * Conventions shared by every call
 *   - Rods are packed one after another ("CSR order"): rod r has n_r elements, n_r + 1
 *     nodes and n_r - 1 Voronoi points.  N = sum(n_r + 1), E = sum(n_r), V = E - n_rods.
 *   - Every per-item vector is stored component-major: x[c * N + j], c = 0, 1, 2.
 *   - Directors: Q[(3a + b) * E + i] is the b-th lab component of director d_{a+1} of element
 *     i; the rows of the director matrix are d1, d2, d3 (proper orthogonal).
 *   - Angular velocities w and couples are in the local (director) frame; positions,
 *     velocities and forces in the lab frame.  SI units.
 *   - Every call returns a rod_status and never aborts.  rod_last_error() returns a
 *     thread-local message for the last failing call of the calling thread.
 *   - The library owns all device memory it allocates; caller buffers are only read or
 *     written during the call (or, for on_device copies, on the system's stream).
 *   - Device errors (non-finite state, a segment longer than the contact grid allows,
 *     a contact table overflow, a bounded wait of the surrogate's tensor-core kernel that ran
 *     out) latch into a device error word that rod_system_step() reports after it
 *     synchronises; rod_system_set_state() clears it.  The device-wide wait of the cooperative
 *     launch that steps a rod longer than a thread block holds cannot stall (a cooperative
 *     launch either runs all its blocks at once or fails to launch, ROD_ERR_CUDA); the
 *     surrogate's fused kernel waits on an mbarrier for its own tensor-core operations, at most
 *     a fixed number of polls, after which it latches the error, drains and ends.
 */
#ifndef ROD_H
#define ROD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rod_system rod_system; /* opaque */

typedef enum {
  ROD_OK = 0,
  ROD_ERR_ARG = -1,       /* invalid argument or description */
  ROD_ERR_CUDA = -2,      /* a CUDA runtime call failed (message has the CUDA error) */
  ROD_ERR_NONFINITE = -3, /* the state became NaN/Inf */
  ROD_ERR_TIMEOUT = -4,   /* a bounded device wait (the surrogate's tensor-core kernel) ran out */
  ROD_ERR_OVERFLOW = -5,  /* contact grid or table capacity exceeded */
  ROD_ERR_STATE = -6      /* call not valid in the current state (e.g. no state set) */
} rod_status;

/* Description of the ensemble (Methods: rho, A, E, G, alpha_c, I, B, S, f, c).
 * All pointers are host pointers; the library copies what it needs during create. */
typedef struct {
  int32_t n_rods;
  const int32_t* n_elem;      /* [n_rods] elements per rod, >= 1 */
  const double* rest_len;     /* [E] element rest lengths (> 0) */
  const double* radius;       /* [n_rods] circular cross-section radius */
  const double* youngs;       /* [n_rods] Young's modulus E */
  const double* shear_mod;    /* [n_rods] shear modulus G */
  const double* density;      /* [n_rods] volumetric density rho */
  double alpha_c;             /* shear correction coefficient (4/3 for a circle) */
  const int8_t* clamp_base;   /* [n_rods] or NULL: 1 = node 0 and element 0 held at the state
                                 given to rod_system_set_state */
  const double* rest_kappa;   /* [3*V] or NULL: rest curvature (local frame) */
  const double* rest_sigma;   /* [3*E] or NULL: rest shear/stretch strain (local frame) */
  double gravity[3];          /* body acceleration (lab) */
  double nu_damp;             /* linear damping: force -nu v and couple -nu (I/A) w per length */
  double stokes_gamma;        /* isotropic drag: force -gamma v per length */
  const double* tip_force;    /* [3*n_rods] or NULL: constant lab force on each rod's last node */
  const double* act_amp;      /* [n_rods] or NULL: base couple A sin(2 pi t / T + phi) about d1 on the
                                 first element not held by the clamp */
  const double* act_period;   /* [n_rods] T > 0 (read when act_amp is set) */
  const double* act_phase;    /* [n_rods] phi (read when act_amp is set) */
  const double* elem_couple;  /* [3*E] or NULL: constant local couple per element */
  void* cuda_stream;          /* cudaStream_t to run on, or NULL for a library-created stream */
  /* magnetic couple of magnetized filaments (Methods, Eq. 2): element couple rl (m x (Q b(t))),
   * b(t) = field_b0 + field_bc cos(field_omega t) + field_bs sin(field_omega t) (lab frame, T) */
  const double* magnetization;  /* [3*E] or NULL: m per unit reference length, local frame (A m) */
  double field_b0[3];
  double field_bc[3];
  double field_bs[3];
  double field_omega;           /* rad/s */
  /* travelling-wave muscle couples (internal, net zero): at interior Voronoi point k of rod r,
   * tau_k = A sin(2 pi t / T - 2 pi s_k / lambda + phi) about local d1, s_k the rest arc length
   * of that point; element i receives tau_{i-1} - tau_i */
  const double* muscle_amp;        /* [n_rods] or NULL: A (N m) */
  const double* muscle_period;     /* [n_rods] T > 0 (s) */
  const double* muscle_wavelength; /* [n_rods] lambda > 0 (m) */
  const double* muscle_phase;      /* [n_rods] phi */
  /* walls: half-spaces n . (x - p - u t) >= r for the node spheres of radius r (the rod's);
   * normal force max(0, wall_k delta - wall_c v_rel . n) n and regularised Coulomb friction
   * -wall_mu f_n v_t / max(|v_t|, wall_vslip) on every penetrating node */
  int32_t n_walls;              /* 0 .. ROD_MAX_WALLS */
  const double* wall_point;     /* [n_walls][3] p (m) */
  const double* wall_normal;    /* [n_walls][3] unit n */
  const double* wall_velocity;  /* [n_walls][3] u (m/s) or NULL (fixed walls) */
  double wall_k, wall_c, wall_mu, wall_vslip;
} rod_system_desc;

#define ROD_MAX_WALLS 8

/* Create a system; validates the description (ROD_ERR_ARG with a message on failure).
 * Rods up to the launch shape's elements per block (at most rod_max_elements_per_rod()) are
 * packed into thread blocks in shared memory; a longer rod (up to 2^24 elements) is stepped by
 * a cooperative launch over the whole GPU with its working arrays in global memory and
 * grid-wide barriers between the stages (same arithmetic; not covered by the adjoint). */
rod_status rod_system_create(const rod_system_desc* desc, rod_system** out);

/* Free the system and all its device memory (NULL is accepted). */
rod_status rod_system_destroy(rod_system* sys);

/* Sizes of the packed arrays. */
rod_status rod_system_sizes(const rod_system* sys, int64_t* n_nodes, int64_t* n_elems, int64_t* n_voronoi);

/* Set the state: x, v [3*N], Q [9*E], w [3*E] in the layout above -- the rod's centreline
 * positions r and velocities v, its director frame Q (rows d1, d2, d3) and the angular
 * velocity w = ax(Q dQ^T/dt) in the local frame, the unknowns of Eq. 1a and Eq. 1b (Methods,
 * "Cosserat rod dynamics"), sampled at the nodes (r, v) and elements (Q, w).  on_device = 0: host
 * pointers, copied synchronously and checked for NaN/Inf on the device after the copy (such a
 * state is rejected with ROD_ERR_ARG and the system then holds no state until the next
 * successful call); on_device = 1: device pointers, copied on the system's stream (the caller
 * keeps them valid until the stream reaches the copy; non-finite values surface as
 * ROD_ERR_NONFINITE from the next step).  Records the clamp values, resets the simulated time
 * to 0 and clears the device error word. */
rod_status rod_system_set_state(rod_system* sys, const double* x, const double* v, const double* Q,
                                const double* w, int on_device);

/* Read the state back: r, v, Q, w of Eq. 1 (Methods, "Cosserat rod dynamics"), same layout and
 * on_device meaning as rod_system_set_state; host copies synchronise. */
rod_status rod_system_get_state(rod_system* sys, double* x, double* v, double* Q, double* w, int on_device);

/* Simulated time of the current state (advanced by dt per step; reset by set_state). */
rod_status rod_system_set_time(rod_system* sys, double t);
rod_status rod_system_get_time(const rod_system* sys, double* t);

/* Advance n_steps position-Verlet steps of size dt (> 0): the multi-stage symplectic scheme with
 * the kinematic constraints enforced after every stage (Results, "Performance-oriented software
 * design"), each step a half kinematic stage (x += dt/2 v, Q <- exp(-dt/2 [w]x) Q), the loads of
 * Eq. 1a and Eq. 1b at the half step (contact included when enabled), the dynamic update of v
 * and w, and the second half kinematic stage.  Enqueued on the system's stream;
 * the call synchronises that stream at the end and returns the device error word
 * (ROD_ERR_NONFINITE / ROD_ERR_OVERFLOW / ROD_ERR_TIMEOUT) if one was raised. */
rod_status rod_system_step(rod_system* sys, int64_t n_steps, double dt);

/* Same as rod_system_step but returns as soon as the work is enqueued; call
 * rod_system_sync() to wait and read the error word. */
rod_status rod_system_step_async(rod_system* sys, int64_t n_steps, double dt);
rod_status rod_system_sync(rod_system* sys);

/* Rod-rod contact (Results, "Fibrous granular materials": a normal spring-dashpot force between
 * touching filaments, found through a hash grid instead of an exhaustive search, Fig. 2e):
 * enable = 0 disables it.  k: spring stiffness (N/m),
 * c: dashpot coefficient (N s/m), cell_size: requested cell edge; the grid uses
 * max(cell_size, 2 r_max + 2 l_max (+ the skin)) where l_max is the longest element of the
 * state given to the next set_state (an element later stretched beyond 2 l_max, less a rounding
 * margin, raises ROD_ERR_OVERFLOW), over
 * the bounding box of that state grown by box_margin (m) on each side (segments leaving it
 * are clamped into the boundary cells, which keeps the pair search exact). */
rod_status rod_system_contact_config(rod_system* sys, int enable, double k, double c, double cell_size);

/* Skin list for the contact search (same forces, fewer candidates per step).  With skin > 0
 * each segment keeps the list of other-rod segments whose distance was within
 * r_a + r_b + skin when the list was built from the cell grid (whose edge grows by the skin);
 * the distance of two segments changes by at most the sum of their endpoints' displacements,
 * so while no node has moved by skin / 2 (m) since the build every touching pair is listed and
 * a step evaluates only the listed pairs.  The step kernels track the largest displacement on
 * the device and the list is rebuilt there when it reaches skin / 2 (no host round trip).
 * Forces are those of the direct search up to the order of summation.  skin = 0 (default):
 * the cell grid is rebuilt and searched at every step.  ROD_ERR_ARG for skin < 0 or not
 * finite.  Takes effect at the next step; the grid is rebuilt. */
rod_status rod_system_contact_skin(rod_system* sys, double skin);

/* Number of skin-list builds since the contact grid was last set up (by set_state, a change of
 * the contact configuration or of the skin): *n = 0 without a skin list.  Synchronises on the
 * system's stream. */
rod_status rod_system_contact_list_builds(rod_system* sys, int64_t* n);

/* Rod-rod friction (Results, "Fibrous granular materials": normal force and friction): at a
 * contact with normal force f_n the tangential force -mu f_n v_t / max(|v_t|, v_slip) acts at
 * the closest points (v_t: the tangential relative velocity), split onto the nodes like the
 * normal force.  mu = 0 turns it off.  ROD_ERR_ARG for mu < 0 or, with mu > 0, v_slip <= 0. */
rod_status rod_system_friction(rod_system* sys, double mu, double v_slip);

/* Right-hand side of Eq. 1a and Eq. 1b (Methods, "Cosserat rod dynamics") at the current state
 * and time t: node accelerations acc_v [3*N] (Eq. 1a divided by the lumped node mass) and
 * element angular accelerations acc_w [3*E] (constraints on rates applied: clamped node 0
 * and element 0 read zero), contact forces included when enabled.  Device pointers. */
rod_status rod_system_rhs(rod_system* sys, double t, double* acc_v, double* acc_w);

/* Contact forces on the nodes [3*N] at the current state (zero when contact is off), the
 * spring-dashpot term of f in Eq. 1a (Results, "Fibrous granular materials"). Device pointer. */
rod_status rod_system_contact_forces(rod_system* sys, double* f);

/* Contact pair set of the current state (Results, "Fibrous granular materials", Fig. 2e: the
 * hash-grid search must find exactly the pairs an exhaustive search finds), for checking the
 * broad phase.  The cell grid is built and searched as in a step without a skin list; every
 * pair of segments (a, b) of different rods, a < b (element indices in CSR order), whose
 * closest-point distance is below r_a + r_b is written to pairs[2k], pairs[2k + 1] for
 * k < cap, in no particular order.  *n_pairs receives the number of such pairs (which may
 * exceed cap: then only cap were written) and *n_candidates, when not NULL, the number of pairs
 * that reached the FP64 evaluation after the grid and the FP32 cull.  pairs: host buffer of
 * 2*cap int64 (may be NULL with cap = 0 to count only).  Synchronises; ROD_ERR_STATE without a
 * state or with contact disabled. */
rod_status rod_system_contact_pairs(rod_system* sys, int64_t* pairs, int64_t cap, int64_t* n_pairs,
                                    int64_t* n_candidates);

/* Launch shape used by the step kernels: elements per thread block and threads per block
 * (0 keeps the built-in default for that value).  Returns ROD_ERR_ARG if the shape cannot
 * fit the block limits or needs more shared memory than a block has (rods longer than the
 * shape's elements per block take the cooperative path). */
rod_status rod_system_set_launch(rod_system* sys, int32_t elems_per_block, int32_t threads_per_block);
rod_status rod_system_get_launch(const rod_system* sys, int32_t* elems_per_block, int32_t* threads_per_block);

/* Energy and frame diagnostics of the current state (Methods: the Cosserat rod of Eq. 1; the
 * energy the explicit symplectic step conserves without damping and loads).  One warp per rod.
 * per_rod: device [9*R] (row c holds component c of every rod) or NULL:
 *   0  translational kinetic energy, sum over the rod's nodes of 1/2 m |v|^2
 *   1  rotational kinetic energy, sum over its elements of 1/2 rho I_c rl w_c^2
 *   2  shear/stretch energy, sum over its elements of 1/2 rl S_c (sigma_c - sigma0_c)^2 with
 *      sigma = Q (x_{i+1} - x_i) / rl - (0, 0, 1) in the element's frame
 *   3  bend/twist energy, sum over its Voronoi points of 1/2 D B_c (kappa_c - kappa0_c)^2 with
 *      kappa = -log(Q_{k+1} Q_k^T) / D, D the mean of the two rest lengths
 *   4  work potential: -sum m g . x over its nodes - F_tip . x_tip
 *   5  largest entry of |Q Q^T - I| over its elements (orthonormality of the directors)
 *   6-8  the position x, y, z of its last node (the tip)
 * totals: host [6] or NULL: rows 0-4 summed over the rods, row 5 maximised (a fixed order: the
 * same bits on every call).  Contact, walls, fields, actuation and damping hold no potential
 * here.  With totals the call synchronises on the system's stream; otherwise it only enqueues
 * (2 kernels with totals, 1 without; counted by rod_system_launch_count).  ROD_ERR_STATE
 * without a state. */
rod_status rod_system_diagnostics(rod_system* sys, double* per_rod, double* totals);

/* How the current launch shape packs the rods into thread blocks: the number of block packs,
 * how many of them list their rods (best-fit-decreasing packs of rods that are not consecutive
 * in index order; the others hold a consecutive run of rods), and the number of rods longer
 * than a block holds (one cooperative launch each).  Any output may be null.  Host-side only:
 * no device work, no synchronisation. */
rod_status rod_system_pack_info(const rod_system* sys, int32_t* n_packs, int32_t* n_listed, int32_t* n_long);

/* The packing rod_system_set_launch makes for elems_per_block = cap_elems and a rods-per-block
 * limit cap_rods, computed on the host (no GPU, no system) for inspection and tests.
 * n_elem [n_rods]: elements per rod (>= 1), rods stored one after another (elements, nodes and
 * Voronoi points numbered rod by rod).  Outputs, each may be null:
 *   n_packs, n_list, n_long: block packs, entries of the rod list, rods longer than cap_elems
 *     (those run one cooperative launch each and are in no block pack);
 *   packs [10 * n_packs], in launch order (heaviest first), per pack: first rod, rods, first
 *     element, elements, first node, nodes, first Voronoi point, Voronoi points (the four
 *     "first" values are the first rod's when the pack lists its rods), listed (0: the rods
 *     first rod .. first rod + rods - 1; 1: the rods of list entries list_off ..), list_off;
 *   list [2 * n_list]: (global rod, the rod's first element within its pack).
 * Call with null packs and list to learn the sizes.  ROD_ERR_ARG for a rod without elements
 * or a capacity below 1. */
rod_status rod_plan_packs(const int32_t* n_elem, int32_t n_rods, int32_t cap_elems, int32_t cap_rods,
                          int32_t* n_packs, int32_t* n_list, int32_t* n_long, int32_t* packs, int32_t* list);

/* Differentiation (hand-written adjoint of the step; rod-rod contact must be off: its state
 * derivatives are not in the reverse sweep; the magnetic couple and walls (normal force and
 * friction, piecewise smooth: derivatives of the active branch) are covered, muscle couples
 * depend on time only).
 * rod_system_set_params replaces the rest curvature [3*V] and/or the element couples [3*E]
 * (NULL leaves one unchanged; on_device as for set_state).
 * rod_system_forward_checkpointed advances n_steps steps of dt from the current state, one
 * step per launch, keeping the state every `every` steps in library memory.
 * rod_system_backward takes the adjoint of the final state (device pointers, layout of the
 * state) and writes the gradients of the loss with respect to the rest curvature [3*V] and
 * the element couples [3*E] (device pointers, overwritten): it recomputes each segment of
 * `every` steps from its checkpoint and runs the adjoint step kernel backwards over it.  The
 * system's state is left at the final state.  Rods longer than one adjoint thread block holds
 * (256 elements with the default shape) are rejected with ROD_ERR_ARG.
 * rod_system_adjoint_of_state copies the adjoint of the initial state of the last backward
 * pass (device pointers). */
rod_status rod_system_set_params(rod_system* sys, const double* rest_kappa, const double* elem_couple, int on_device);
rod_status rod_system_forward_checkpointed(rod_system* sys, int64_t n_steps, double dt, int32_t every);
rod_status rod_system_backward(rod_system* sys, const double* adj_x, const double* adj_v, const double* adj_Q,
                               const double* adj_w, double* grad_rest_kappa, double* grad_elem_couple);
rod_status rod_system_adjoint_of_state(rod_system* sys, double* adj_x, double* adj_v, double* adj_Q, double* adj_w);

/* With contact, rod_system_step replays a CUDA graph of 32 captured steps (captured on an
 * internal stream, launched on the system's stream) unless profiling is on or a rod is longer
 * than a block holds; enable = 0 makes every step an eager sequence of launches (same kernels,
 * same results).  With the skin list the rebuild kernels sit in a conditional node of the graph
 * that the device-side rebuild decision opens only when a rebuild is due.  A captured graph is
 * kept while nothing it bakes in changes (step parameters, dt, launch shape, contact grid and
 * constants); otherwise the next step call captures a new one. */
rod_status rod_system_set_graphs(rod_system* sys, int enable);

/* Per-kernel timing (tracing): enable = 1 records a CUDA event pair on the system's stream
 * around every kernel launch and resets the totals; enable = 0 stops recording. */
rod_status rod_system_profile(rod_system* sys, int enable);

/* Number of kernel classes reported by rod_system_profile_read. */
int32_t rod_profile_classes(void);

/* Accumulated device time (ms, from the event pairs) and launch count of kernel class k
 * (0 <= k < rod_profile_classes()); *name receives a static string.  Synchronises on the
 * recorded events. */
rod_status rod_system_profile_read(rod_system* sys, int32_t k, const char** name, double* total_ms,
                                   int64_t* launches);

/* Total number of kernels this system has launched since it was created, those of replayed
 * graphs included (rebuild kernels of a graph's conditional node count when they ran: with a
 * skin list the call reads a device counter and synchronises on the system's stream). */
rod_status rod_system_launch_count(const rod_system* sys, int64_t* launches);

/* Autotuner: time trial_steps steps of dt (after one warm-up step) for every valid launch shape
 * (elements per block 192..768, threads per block 128..512), keep the fastest and restore the
 * state and time.  Results are cached per ensemble signature (rod count, elements, longest and
 * shortest rod, contact on/off) for the process, and in the text file named by the environment
 * variable ROD_AUTOTUNE_CACHE when it is set.  Outputs may be NULL; *best_ms is the time per
 * step of the winner (-1 when it came from the cache). */
rod_status rod_system_autotune(rod_system* sys, double dt, int32_t trial_steps, int32_t* best_elems,
                               int32_t* best_threads, double* best_ms);

/* Longest rod (elements) one thread block can hold with the largest supported shape; longer
 * rods take the cooperative path. */
int32_t rod_max_elements_per_rod(void);

/* Learned surrogate of a window of fine steps for rods of 50 elements (the paper has no
 * learned component): four 1D convolutions along the rod (kernel 5, 64 channels, SiLU), BF16
 * weights and activations on tensor cores with FP32 accumulation, FP64 state update.
 * Inputs per node position j (24 features; feature = float(raw - in_shift) * in_scale, zero
 * where undefined): position minus the base node [0..2], velocity [3..5], directors d1, d2 of
 * element j [6..11], angular velocity of element j [12..14], half the axial vector of
 * R - R^T with R = Q_j Q_{j-1}^T [15..17], the edge Q_j (x_{j+1} - x_j) [18..20] and the base
 * couple A sin(2 pi t / T + phi) at the window's start, middle and end [21..23].
 * Outputs (15 channels): the change of x, v, d1, d2, w over the window minus the kinematic
 * prior (x + T v; Q turned by exp([-T w]x); v and w unchanged), divided by out_scale.  The
 * update is state = prior + out_scale * output in FP64, then Gram-Schmidt on d1, d2 with
 * d3 = d1 x d2; a clamped rod keeps node 0 and element 0 (at rest).
 *   create(window_steps, dt)        a network with all parameters zero for windows of
 *                                   window_steps fine steps of dt (T = window_steps * dt)
 *   num_params()                    length of the FP32 parameter vector
 *   set_params / get_params         FP32 parameters (host or device); set resets Adam's moments
 *   set_scales(shift[24], scale[24], out[15])   feature shift / scale and output scales (host)
 *   set_prior(flags)                the form of the update: bit 0 positions get the prior
 *                                   x + T v (else x), bit 1 directors exp([-T w]x) Q (else Q),
 *                                   bit 2 velocities are the output alone (else v + output),
 *                                   bit 3 angular velocities are the output alone (else w +
 *                                   output); default 3.  Targets follow the same form.
 *   train_step(...)                 one Adam step (lr > 0) or loss + gradient only (lr <= 0) on a
 *                                   batch of windows: states at the window start and end for
 *                                   nwin rods in the system layout (device pointers), act
 *                                   [3][nwin] = base couple at the window's start, middle and
 *                                   end; *loss_out (host, optional) receives the mean-square
 *                                   loss over nwin x 51 x 15 outputs (synchronises the stream)
 *   get_grad                        the FP32 gradient of the last train_step
 *   raw_features                    the unscaled FP64 features [nwin][24][51] (device) and a mask
 *                                   [nwin][24][51] (int8, 1 where defined; NULL to skip)
 *   raw_targets                     the unscaled FP64 targets [nwin][15][51] (device): state
 *                                   change over the window minus the prior
 *   forward                         raw outputs [nwin][51][16] (FP32, device) for given states
 *   apply(sys, n_calls)             advance every rod of a system (50 elements each, contact
 *                                   off) by n_calls windows; synchronises the system's stream
 *   rollout(sys, shadow, ...)       n_calls windows with a periodic check: every check_every
 *                                   calls the tips of the sampled rods sample_rods[0..n_sample)
 *                                   are compared with the shadow system, which holds those rods
 *                                   (same order, same time) and follows them with the plain
 *                                   step; if max |x_tip - x_tip(shadow)| / L exceeds bound, the
 *                                   segment is undone and redone with the plain step.  stats
 *                                   (optional) receives the counts and errors.
 *   rollout_local(sys, shadows, n_shadows, ...)   the same with local checks: segment k's check
 *                                   restarts the plain step from the surrogate's state of the
 *                                   sampled rods at the segment's start (on shadow k mod
 *                                   n_shadows, each holding the n_sample rods) and compares the
 *                                   tips at its end; up to n_shadows (1..8) checks run while the
 *                                   network goes on; a segment above its share of the bound
 *                                   (bound x its calls / check_every) is undone with every later
 *                                   one and redone with the plain step.  Segments have
 *                                   check_every calls except toward the end, where each has about
 *                                   a third of the calls after it (at least one), so that the
 *                                   last checks end soon after the network does.
 * All calls return ROD_ERR_ARG for bad arguments, ROD_ERR_CUDA for CUDA failures. */
typedef struct rod_surrogate rod_surrogate;
typedef struct {
  int64_t surrogate_calls;   /* windows advanced by the network */
  int64_t fallback_calls;    /* windows redone with the plain step */
  int64_t checks;            /* error checks made */
  double max_err;            /* largest sampled error kept (after any fallback) */
  double last_err;           /* sampled error at the end */
  double rejected_err;       /* largest sampled error that caused a fallback (0: none) */
  double sum_err;            /* sum of the accepted checks' errors (rollout_local: a bound on the
                                accumulated error when segment errors add up without growth) */
} rod_surrogate_stats;
rod_status rod_surrogate_create(int32_t window_steps, double dt, rod_surrogate** out);
rod_status rod_surrogate_destroy(rod_surrogate* sur);
int64_t rod_surrogate_num_params(void);
rod_status rod_surrogate_set_params(rod_surrogate* sur, const float* params, int on_device);
rod_status rod_surrogate_get_params(rod_surrogate* sur, float* params, int on_device);
rod_status rod_surrogate_set_scales(rod_surrogate* sur, const double* in_shift, const double* in_scale,
                                    const double* out_scale);
rod_status rod_surrogate_set_prior(rod_surrogate* sur, int32_t flags);
rod_status rod_surrogate_train_step(rod_surrogate* sur, const double* x0, const double* v0, const double* Q0,
                                    const double* w0, const double* x1, const double* v1, const double* Q1,
                                    const double* w1, const double* act, int32_t nwin, float lr, float* loss_out,
                                    void* cuda_stream);
rod_status rod_surrogate_get_grad(rod_surrogate* sur, float* grad, int on_device);
/* Intermediate arrays of the last rod_surrogate_train_step, copied to the host as FP32 (BF16
 * arrays widened exactly), so that each layer of the kernels can be checked on its own; a test
 * hook with no counterpart in the paper.  Rows are positions + 2 (rows 0, 1 and 53..63 are the
 * convolutions' zero padding), windows outermost, channels innermost.  which:
 *   0       network input (features)       [nwin][64][32]  BF16
 *   1..3    hidden activations of layer 1..3 [nwin][64][64] BF16
 *   4..6    pre-activations of layer 1..3   [nwin][64][64]  FP32
 *   7       network output                  [nwin][51][16]  FP32
 *   8       training targets                [nwin][51][16]  FP32
 *   9       loss gradient of the output     [nwin][64][16]  BF16
 *   10..12  back-propagated gradients at the outputs of layers 3, 2, 1 [nwin][64][64] BF16
 * cap: room in out (floats); *n_out receives the element count (cap = 0: count only).
 * ROD_ERR_STATE before the first training step.  Synchronises the device. */
rod_status rod_surrogate_debug_buffer(rod_surrogate* sur, int32_t which, float* out, int64_t cap, int64_t* n_out);
rod_status rod_surrogate_forward(rod_surrogate* sur, const double* x, const double* v, const double* Q,
                                 const double* w, const double* act, int32_t nwin, float* out, void* cuda_stream);
rod_status rod_surrogate_raw_features(rod_surrogate* sur, const double* x, const double* v, const double* Q,
                                      const double* w, const double* act, int32_t nwin, double* out, int8_t* mask,
                                      void* cuda_stream);
rod_status rod_surrogate_raw_targets(rod_surrogate* sur, const double* x0, const double* v0, const double* Q0,
                                     const double* w0, const double* x1, const double* v1, const double* Q1,
                                     const double* w1, int32_t nwin, double* out, void* cuda_stream);
/* Noise-injected training-window start (the surrogate's training, which perturbs each window's
 * start so that the network learns to contract perturbations; the paper has no counterpart).
 *   x0, v0, Q0, w0  device window starts of nwin rods of 50 elements ([3][nwin 51], [3][nwin 51],
 *                   [9][nwin 50], [3][nwin 50])
 *   rx, rv, rw, ra  device standard normal draws shaped like x, v, w, w (may be NULL when noise = 0)
 *   spread          host double [15]: the output scales of the 15 state channels
 *   noise           >= 0; positions, velocities and angular velocities move by noise x their
 *                   channel's spread x the draw, the directors d1, d2 turn by the lab-frame
 *                   angle vector noise x (largest director spread) x ra to first order and are
 *                   re-orthonormalised (Gram-Schmidt, d3 = d1 x d2); noise = 0 only
 *                   re-orthonormalises the directors
 *   held            device int8 [nwin] (NULL: none): a held window keeps node 0's position and
 *                   element 0's directors, with zero velocity and angular velocity there
 *   x, v, Q, w      device outputs, shaped like the inputs and not overlapping them
 * Asynchronous on cuda_stream.  ROD_ERR_ARG for a bad argument or a non-finite spread. */
rod_status rod_surrogate_perturb(rod_surrogate* sur, const double* x0, const double* v0, const double* Q0,
                                 const double* w0, int32_t nwin, const double* rx, const double* rv, const double* rw,
                                 const double* ra, const double* spread, double noise, const int8_t* held, double* x,
                                 double* v, double* Q, double* w, void* cuda_stream);
rod_status rod_surrogate_apply(rod_surrogate* sur, rod_system* sys, int64_t n_calls);
/* Polls of the fused inference kernel's waits for its tensor-core MMAs before it gives up
 * (0: the default, 2^20).  A wait that runs out latches ROD_ERR_TIMEOUT into the system's error
 * word (returned by rod_surrogate_apply and the system's next step or sync).  A test hook: with
 * the top bit set the kernel issues no MMA, so its first wait runs out after the remaining
 * bits' polls and the kernel ends without updating the state. */
rod_status rod_surrogate_set_wait_polls(rod_surrogate* sur, uint32_t polls);
/* One window call of the fused inference kernel with every layer's arrays captured, for
 * checking the tensor-core layers element by element (a test hook; the paper has no
 * counterpart).  pre, act: host buffers of cap >= 4 * R * 51 * 64 floats; entry
 * ((l * R + b) * 51 + p) * 64 + o receives, for layer l = 0..3, rod b, node position p and
 * output channel o, the FP32 accumulator plus bias (pre; the output layer fills o < 16), and
 * the BF16 input of layer l, widened (act; l = 0: the features, channels 0..31).  Advances the
 * system by one window like rod_surrogate_apply(sur, sys, 1).  ROD_ERR_STATE when the unfused
 * path is forced (ROD_SURROGATE_UNFUSED). */
rod_status rod_surrogate_apply_debug(rod_surrogate* sur, rod_system* sys, float* pre, float* act, int64_t cap);
rod_status rod_surrogate_rollout(rod_surrogate* sur, rod_system* sys, rod_system* shadow, const int32_t* sample_rods,
                                 int32_t n_sample, int64_t n_calls, int32_t check_every, double bound,
                                 rod_surrogate_stats* stats);
rod_status rod_surrogate_rollout_local(rod_surrogate* sur, rod_system* sys, rod_system* const* shadows,
                                       int32_t n_shadows, const int32_t* sample_rods, int32_t n_sample,
                                       int64_t n_calls, int32_t check_every, double bound,
                                       rod_surrogate_stats* stats);

/* Contact forces without allocating anything (the paper has no counterpart: this is a service
 * for callers that cannot allocate device memory when they need the forces, such as code
 * running inside another framework's allocator or memory pool, or a loop that must not enter
 * the driver's allocator).  All temporaries live in one fixed file-scope device array of
 * about 16 MB (sized by the two limits below) that every GPU loading the library holds until
 * the process exits.
 *   n_rods    number of rods (> 0)
 *   node_off  device int32 [n_rods + 1]: CSR node offsets, node_off[0] = 0, rod r owns nodes
 *             node_off[r] .. node_off[r+1]-1 (at least 2 nodes); elements = nodes - n_rods
 *   radius    device double [n_rods]
 *   x, v      device double [3 * N], component-major node positions and velocities
 *   k, c      spring stiffness and dashpot coefficient (finite, >= 0)
 *   cell_size requested cell edge; the grid uses max(cell_size, 2 r_max + l_max) of these positions,
 *             grown (which keeps the search exact) until the grid over the midpoints' bounding
 *             box has at most ROD_NOALLOC_MAX_CELLS cells
 *   f         device double [3 * N] output, overwritten with the contact force on every node
 *   cuda_stream  stream to run on (NULL = legacy default stream)
 * The same forces as rod_system_contact_forces for the same state (pair set exact, sums in
 * another order).  More than ROD_NOALLOC_MAX_SEGMENTS elements -> ROD_ERR_OVERFLOW before any
 * launch; a cell with more than 512 segments -> ROD_ERR_OVERFLOW; non-finite positions ->
 * ROD_ERR_NONFINITE.  The call synchronises the stream before it returns.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), so make it before any
 * stream capture.  Every call shares the array and finds the previous call's contents in it
 * (what must start at zero is cleared); calls that overlap on the GPU race on it. */
#define ROD_NOALLOC_MAX_SEGMENTS 131072
#define ROD_NOALLOC_MAX_CELLS 524288
rod_status rod_contact_forces_noalloc(int32_t n_rods, const int32_t* node_off, const double* radius, const double* x,
                                      const double* v, double k, double c, double cell_size, double* f,
                                      void* cuda_stream);

/* Thread-local message of the last failing call. */
const char* rod_last_error(void);

/* Library version string. */
const char* rod_version(void);

#ifdef __cplusplus
}
#endif
#endif
