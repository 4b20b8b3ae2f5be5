// rod_step.cu -- FP64 step kernels of the discrete Cosserat-rod method for sm_103a.
//
// One thread block owns a "pack" of consecutive rods (CSR order) and stages their nodes,
// directors and work arrays in shared memory, so that the difference (Delta^h) and averaging
// (A^h) operators of Eq. 1 read their neighbours on chip; ghost values at the rod ends are the
// zeros of the discrete operators.  Without contact the rods are independent, so a block runs
// all requested steps on chip and touches HBM once per launch (the paper's asynchronous
// protocol taken to the whole step loop).  With contact a launch performs one step and the
// contact forces come from the cell-list kernels.
//
// The FP64 pipe of this part (2 DFMA/clk/SM) bounds the step, so the kernel avoids FP64
// divisions (precomputed reciprocals of constants, one rsqrt per element, one reciprocal per
// Voronoi point) and evaluates the rotation exponential and logarithm of small angles by
// their Taylor series in theta^2 (no sqrt, no sin/cos/atan2 on the common path); large
// angles fall back to sincos/atan2.
//
// Step (position Verlet, Results "Performance-oriented software design"): half kinematic
// stage, dynamic stage at t + dt/2, half kinematic stage; kinematic constraints after every
// stage.  The second half stage of step s and the first of step s+1 are fused into one
// kinematic update of dt (exp(-h w) exp(-h w) = exp(-2h w) for a fixed w).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "rod_internal.h"
#include "rod_step_device.cuh"

namespace rod {

namespace {

// ------------------------------------------------------------------------- the pack kernel

template <int MODE>
__global__ void __launch_bounds__(512) pack_kernel(StepParams P, LaunchShape S, int64_t n_steps, double t0, double dt,
                                                   int last_half, double* acc_v, double* acc_w) {
  extern __shared__ double smem_d[];
  // a step after a latched error (non-finite state, contact overflow) is skipped
  if (MODE == MODE_ONE_STEP && *(volatile int*)P.err != 0) return;
  const Pack pk = P.packs[blockIdx.x];
  Smem m = carve(smem_d, S);
  const int Ep = pk.nelem, Np = pk.nnode;

  stage_pack(P, pk, m);

  if (MODE == MODE_KIN_HALF) {
    kinematic(P, pk, m, 0.5 * dt);
    __syncthreads();
  } else if (MODE == MODE_RHS) {
    actuation_values(P, pk, m, t0);
    stage_elements(P, pk, m);
    __syncthreads();
    stage_voronoi(P, pk, m);
    __syncthreads();
    stage_rotation<MODE_RHS>(P, pk, m, dt, 0.0, acc_w);
    stage_translation<MODE_RHS>(P, pk, m, dt, acc_v, t0);
    return;
  } else {
    if (MODE == MODE_STEPS) {
      kinematic(P, pk, m, 0.5 * dt);
      __syncthreads();
    }
    const double tbase = P.t_dev ? *P.t_dev : t0;
    const bool timed = has_time_values(P);
    if (n_steps > 0) actuation_values(P, pk, m, tbase + 0.5 * dt);
    for (int64_t s = 0; s < n_steps; ++s) {
      stage_elements(P, pk, m);
      __syncthreads();
      stage_voronoi(P, pk, m);
      __syncthreads();
      // rate updates fused with the following kinematic stage: each thread moves only the
      // elements and nodes whose rates it has just updated
      const bool last = (s == n_steps - 1);
      const double h = (last && (MODE == MODE_STEPS || last_half)) ? 0.5 * dt : dt;
      const double t = tbase + (static_cast<double>(s) + 0.5) * dt;
      stage_rotation<MODE_STEPS>(P, pk, m, dt, h, nullptr);
      stage_translation<MODE_STEPS>(P, pk, m, dt, nullptr, t, h);
      // the next step's time values: their only readers (the element stage) are past a barrier;
      // the next step's element stage waits for the barrier below
      if (timed && !last) time_values(P, pk, m, t + dt);
      __syncthreads();
    }
  }

  // ---- contact binning of the positions this launch leaves behind (the next step's
  // half-step positions): FP32 midpoint, half length and cell of every segment, counted per
  // cell with one atomic per distinct cell in the warp.
  if ((MODE == MODE_KIN_HALF || (MODE == MODE_ONE_STEP && !last_half)) && P.bin_count) {
    bool grid_bad = false, nonfinite = false;
    for (int i = threadIdx.x; i < Ep; i += blockDim.x) {
      const int j = i + m.erod[i];
      float p0[3], p1[3], mid[3];
      float ll = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        p0[c] = static_cast<float>(m.X[c * m.CN + j]);
        p1[c] = static_cast<float>(m.X[c * m.CN + j + 1]);
        mid[c] = 0.5f * (p0[c] + p1[c]);
        ll = fmaf(p1[c] - p0[c], p1[c] - p0[c], ll);
      }
      const float len = sqrtf(ll);
      const bool fin = isfinite(mid[0]) && isfinite(mid[1]) && isfinite(mid[2]) && isfinite(len);
      nonfinite |= !fin;
      grid_bad |= fin && !(len <= P.bin_l_allowed);
      int ic[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float q = floorf((mid[c] - P.bin_lo[c]) * P.bin_inv_h);
        q = fminf(fmaxf(q, 0.f), static_cast<float>(P.bin_dim[c] - 1));
        ic[c] = static_cast<int>(q);
      }
      const int cell = (ic[2] * P.bin_dim[1] + ic[1]) * P.bin_dim[0] + ic[0];
      const int ge = pk.elem0 + i;
      P.bin_cell[ge] = cell;
      P.bin_prox[ge] = make_float4(mid[0], mid[1], mid[2], 0.5f * len);
      const unsigned peers = __match_any_sync(__activemask(), cell);
      if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(P.bin_count + cell, __popc(peers));
    }
    if (nonfinite) atomicOr(P.err, ERR_NONFINITE);
    if (grid_bad) atomicOr(P.err, ERR_GRID);
  }

  // ---- write back, flag non-finite values
  bool bad = false;
  for (int i = threadIdx.x; i < Ep; i += blockDim.x) {
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double q = m.QQ[a * m.CE + i];
      bad |= !isfinite(q);
      P.Q[a * P.E + pk.elem0 + i] = q;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double ww = m.WW[c * m.CE + i];
      bad |= !isfinite(ww);
      P.w[c * P.E + pk.elem0 + i] = ww;
    }
  }
  for (int j = threadIdx.x; j < Np; j += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double xx = m.X[c * m.CN + j], vv = m.VN[c * m.CN + j];
      bad |= !isfinite(xx) || !isfinite(vv);
      P.x[c * P.N + pk.node0 + j] = xx;
      P.v[c * P.N + pk.node0 + j] = vv;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(P.err, ERR_NONFINITE);
}

}  // namespace

size_t step_smem_bytes(const LaunchShape& s) {
  const size_t CE = s.cap_elems, CR = s.cap_rods, CN = CE + CR, CV = CE;
  const size_t doubles = 3 * CN + 3 * CN + 9 * CE + 3 * CE + 3 * CE + 3 * CE + CE + CE + 3 * CV + 3 * CV + CE + CN + CR + 4;
  const size_t ints = CR + 1;
  const size_t shorts = CE + CN + CV;
  return doubles * sizeof(double) + ints * sizeof(int) + shorts * sizeof(short) + 16;
}

const char* kernel_class_name(int k) {
  static const char* names[K_NUM_CLASSES] = {"pack_steps", "pack_one_step", "kin_half", "rhs", "contact_bin",
                                             "contact_scan", "contact_scatter", "contact_sort", "contact_gather",
                                             "contact_node_forces", "misc"};
  return (k >= 0 && k < K_NUM_CLASSES) ? names[k] : "?";
}

cudaError_t launch_pack_kernel(const StepParams& P, const LaunchShape& s, int mode, int64_t n_steps, double t0,
                               double dt, int last_half, double* acc_v, double* acc_w, cudaStream_t st,
                               const LaunchHook& hook) {
  const size_t smem = step_smem_bytes(s);
  const dim3 grid(P.n_packs), block(s.threads);
  const int cls = mode == MODE_STEPS ? K_PACK_STEPS : mode == MODE_ONE_STEP ? K_PACK_ONE_STEP
                : mode == MODE_KIN_HALF ? K_KIN_HALF : K_RHS;
  hook.before(cls, st);
  struct After {
    const LaunchHook& h; int c; cudaStream_t s;
    ~After() { h.after(c, s); }
  } after_guard{hook, cls, st};
  switch (mode) {
    case MODE_STEPS: {
      cudaFuncSetAttribute(pack_kernel<MODE_STEPS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      pack_kernel<MODE_STEPS><<<grid, block, smem, st>>>(P, s, n_steps, t0, dt, last_half, acc_v, acc_w);
      break;
    }
    case MODE_ONE_STEP: {
      cudaFuncSetAttribute(pack_kernel<MODE_ONE_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      pack_kernel<MODE_ONE_STEP><<<grid, block, smem, st>>>(P, s, n_steps, t0, dt, last_half, acc_v, acc_w);
      break;
    }
    case MODE_KIN_HALF: {
      cudaFuncSetAttribute(pack_kernel<MODE_KIN_HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      pack_kernel<MODE_KIN_HALF><<<grid, block, smem, st>>>(P, s, n_steps, t0, dt, last_half, acc_v, acc_w);
      break;
    }
    case MODE_RHS: {
      cudaFuncSetAttribute(pack_kernel<MODE_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      pack_kernel<MODE_RHS><<<grid, block, smem, st>>>(P, s, n_steps, t0, dt, last_half, acc_v, acc_w);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace rod
