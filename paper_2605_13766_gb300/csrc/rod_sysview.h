// rod_sysview.h -- access to a system's device state for the surrogate (internal to librod).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/rod.h"
#include "rod_internal.h"

namespace rod {

struct SysView {
  double *x, *v, *Q, *w;   // device state (component-major)
  int64_t N, E;
  int R, max_n, min_n;
  const RodConst* rods;    // device per-rod constants
  const double* rest_len;  // device rest length per element
  bool contact;            // rod-rod contact enabled
  int n_packs;             // thread blocks of one step launch
  cudaStream_t stream;
  double* t;               // the system's simulated time (host)
  int* err;                // the system's device error word
};

rod_status system_view(rod_system* sys, SysView* out);

// Clear a system's latched device error word (on its stream), e.g. after a shadow copy of
// rods ran into non-finite values; returns the CUDA status of the enqueue.
cudaError_t system_clear_error(rod_system* sys);

}  // namespace rod
