// rod_contact.h -- rod-rod contact pipeline of librod (uniform cell list + narrow phase).
// Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/rod.h"
#include "rod_internal.h"

namespace rod {

// Device-side control of the skin list: the largest squared node displacement since the last
// build (bits of a non-negative double, raised by the step kernels), the rebuild decision of
// the current evaluation, and a request to rebuild from the host.
struct ListCtl {
  unsigned long long disp2;
  int gate;
  int force;
  int builds;  // list builds since the grid was set up
  int opened;  // rebuilds that ran inside a replayed graph's conditional node (launch accounting)
  int n_active;  // segments with candidates at the last build (entries of ContactState::active)
};

// Kernels of one skin-list rebuild (bin, scan x3, fill, scatter, sort, records, build, active
// set, snapshot).
constexpr int kListRebuildKernels = 11;

// Capacity of one segment's candidate list; a segment with more candidates scans its
// neighbourhood of the last build instead.  Thick rods cut into short segments give a touching
// segment many candidates (two parallel rods of radius r and element length l: about
// 2 sqrt((2r + skin)^2 - (2r)^2) / l on each neighbour), hence room for 32.
constexpr int kNbrCap = 32;

struct ContactState {
  bool enabled = false;
  double k = 0.0, c = 0.0, cell_size = 0.0;
  double mu = 0.0, vslip = 0.0;  // regularised Coulomb friction (mu = 0: none)
  bool grid_valid = false;
  // grid over segment midpoints; midpoints outside are clamped into the boundary cells
  double lo[3] = {0, 0, 0};
  double h = 0.0, inv_h = 0.0;
  int dim[3] = {0, 0, 0};
  int64_t ncell = 0, cap_cells = 0;
  double l_allowed = 0.0;  // longest element the cell size covers (less the FP32 binning margin)
  int version = 0;         // bumped whenever the grid, the constants or a buffer changes
  std::vector<uint64_t> signature;  // what the last version was made of
  int64_t E = 0;
  // device buffers (library-owned)
  int* seg_rod = nullptr;     // [E] rod of each segment
  int* seg_cell = nullptr;    // [E]
  int* cell_count = nullptr;  // [cap_cells + 1]
  int* cell_start = nullptr;  // [cap_cells + 1]
  int* cell_fill = nullptr;   // [cap_cells]
  int* block_sums = nullptr;  // scan scratch
  int64_t n_block_sums = 0;
  int* sorted = nullptr;      // [E] segments ordered by cell, ascending index within a cell
  float4* prox = nullptr;     // [E] FP32 midpoint + half length (culling only)
  float4* recA = nullptr;     // [E] prox in cell order
  int4* recB = nullptr;       // [E] (segment, rod, FP32 radius bits, end of the rod's run) in cell order
  float4* recC = nullptr;     // [E] FP32 half edge (x_{i+1} - x_i) / 2 in cell order
  double* fseg = nullptr;     // [6E] force on the first / second node of each segment
  // skin list (skin > 0): candidates within r_a + r_b + skin at the last build, kept while no
  // node has moved by skin / 2 since (then no pair outside the list can touch)
  double skin = 0.0;
  int sm_count = 0;
  int64_t N = 0;
  int* nbr = nullptr;         // [kNbrCap * E] entry-major: candidate k of segment a at k E + a
  int* nbr_count = nullptr;   // [E] (> kNbrCap: overflowed, scan instead)
  int* slot_of = nullptr;     // [E] slot of each segment in the last build's cell order
  float* x_ref = nullptr;     // [3N] positions of the last build, rounded to FP32
  float4* seg_prox = nullptr; // [2E] FP32 proxies of the current positions, written by the step kernels
  // segments with candidates at the last build (only they can have a contact force until the
  // next one): a bit per segment index and the compact list the force kernel walks
  unsigned* active_mask = nullptr;  // [(E + 31) / 32]
  int* active = nullptr;            // [E], ctl->n_active entries in use
  ListCtl* ctl = nullptr;
  unsigned long long* bounds = nullptr;  // [8] grid set-up: bounding box, longest segment (order keys)
  bool ctl_live = false;       // ctl holds counts of the current grid
  int64_t opened_before = 0;   // ctl->opened of earlier grids (launch accounting)
};

// Rebuild kernels launched so far inside replayed graphs (reads the device counter).
int64_t contact_list_graph_rebuild_launches(const ContactState& cs, cudaStream_t st);

void contact_release(ContactState& cs);

// Build the grid (once per state / configuration) from the current positions.
rod_status contact_prepare(ContactState& cs, const std::vector<RodConst>& rods_h, const RodConst* rods_dev,
                           const double* x_dev, int64_t N, int64_t E, int R, cudaStream_t st, const LaunchHook& hook);

// Record an error message for rod_last_error() (defined with the ABI) and return st.
rod_status internal_fail(rod_status st, const char* what, const char* detail);

// Enqueue one evaluation of the contact forces at positions x, velocities v -> cs.fseg.
// prebinned: the step kernel already binned these positions (cs.seg_cell, cs.prox and the
// counts); otherwise the counts are cleared and the segments binned here.
cudaError_t contact_compute(ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                            int64_t E, int R, int* err, cudaStream_t st, const LaunchHook& hook, bool prebinned);

// Point the step kernel's binning epilogue at this grid; zero the per-cell counts.
void contact_bin_params(const ContactState& cs, StepParams& P);
cudaError_t contact_clear_counts(const ContactState& cs, cudaStream_t st);

// Skin-list evaluation of the contact forces at x, v -> cs.fseg: rebuild (bin, sort, list) on
// the device when the displacement since the last build reaches skin / 2 or a rebuild was
// requested, then the forces of the listed pairs.  The per-cell counts must be zero on entry
// (contact_clear_counts) and are zero again after a rebuild.
cudaError_t contact_list_compute(ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                                 int64_t E, int R, int* err, cudaStream_t st, const LaunchHook& hook);
// The same in three parts, for graph capture: the decision (with a conditional handle it also
// sets the condition of the graph node that holds the rebuild), the gated rebuild kernels, and
// the forces of the listed pairs.
cudaError_t contact_list_decide(ContactState& cs, cudaStream_t st, const LaunchHook& hook,
                                const cudaGraphConditionalHandle* cond);
cudaError_t contact_list_rebuild(ContactState& cs, const double* x, const RodConst* rods, int64_t N, int64_t E,
                                 int* err, cudaStream_t st, const LaunchHook& hook);
cudaError_t contact_list_force(ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                               int64_t E, int* err, cudaStream_t st, const LaunchHook& hook);
// Point the step kernels' displacement tracking at the list's reference positions.
void contact_list_params(const ContactState& cs, StepParams& P);
// Make the next list evaluation rebuild (after anything that overwrote the cell structures).
cudaError_t contact_list_invalidate(const ContactState& cs, cudaStream_t st);

// Pair set of positions x by the cell-grid search (debug / parity entry point): the pairs (a, b),
// a < b, in contact go to out[2k], out[2k + 1] for k < cap; counts[0] = pairs in contact,
// counts[1] = candidate pairs that passed the FP32 cull (device words, overwritten).
cudaError_t contact_pairs(ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                          int64_t E, int* err, unsigned long long* counts, int64_t* out, int64_t cap, cudaStream_t st,
                          const LaunchHook& hook);

// Sum cs.fseg into node forces f [3N] (debug / parity entry point).
cudaError_t contact_node_forces(const ContactState& cs, const RodConst* rods, int64_t N, int64_t E, int R, double* f,
                                cudaStream_t st, const LaunchHook& hook);

}  // namespace rod
