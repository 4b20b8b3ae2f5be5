// rod_diag.h -- energy and frame diagnostics kernels (internal to librod).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "rod_internal.h"

namespace rod {

struct DiagArgs {
  const double *x, *v, *Q, *w;  // device state, component-major
  const double* rest_len;       // [E]
  const double* inv_m;          // [N] 1 / node mass
  const double* rest_sigma;     // [3][E] or null
  const double* rest_kappa;     // [3][V] or null
  const RodConst* rods;         // [R]
  int64_t N, E, V;
  int R;
  double gravity[3];            // zero when the system has none
  double* per_rod;              // [9][R] output: five energy parts, orthonormality, tip x, y, z
};

// Per-rod rows into A.per_rod (one warp per rod).
cudaError_t launch_diag_rows(const DiagArgs& A, cudaStream_t st);
// The six totals of the rows (device [6]): rows 0-4 summed, row 5 maximised, in a fixed order.
cudaError_t launch_diag_totals(const double* per_rod, int R, double* totals_dev, cudaStream_t st);

}  // namespace rod
