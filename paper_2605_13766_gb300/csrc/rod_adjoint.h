// rod_adjoint.h -- launcher of the adjoint step kernel (internal to librod).
#pragma once
#include <cuda_runtime.h>

#include "rod_internal.h"

namespace rod {

struct AdjointParams {
  StepParams P;       // forward parameters; P.x/v/Q/w point at the step's start state
  double* ax;         // [3N] adjoint of the end state in, of the start state out
  double* av;         // [3N]
  double* aQ;         // [9E]
  double* aw;         // [3E]
  double* g_kappa0;   // [3V] accumulated gradient w.r.t. rest curvature
  double* g_couple;   // [3E] accumulated gradient w.r.t. element couples
  double t;           // time of the start state
  double dt;
  int64_t fwd_smem_doubles;  // size of the forward stages' shared-memory region (doubles)
};

size_t adjoint_smem_bytes(const LaunchShape& s);
cudaError_t launch_adjoint_kernel(const AdjointParams& A, const LaunchShape& s, cudaStream_t st);

}  // namespace rod
