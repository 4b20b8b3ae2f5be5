// rod_contact.h -- rod-rod contact pipeline of librod (uniform cell list + narrow phase).
// Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/rod.h"
#include "rod_internal.h"

namespace rod {

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
  int version = 0;         // bumped whenever the grid is rebuilt
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
  int4* recB = nullptr;       // [E] (segment, rod, FP32 radius bits, 0) in cell order
  double* fseg = nullptr;     // [6E] force on the first / second node of each segment
};

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

// Sum cs.fseg into node forces f [3N] (debug / parity entry point).
cudaError_t contact_node_forces(const ContactState& cs, const RodConst* rods, int64_t N, int64_t E, int R, double* f,
                                cudaStream_t st, const LaunchHook& hook);

}  // namespace rod
