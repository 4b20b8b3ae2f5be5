// rod_step.cu -- FP64 step kernels of the discrete Cosserat-rod method for sm_103a.
//
// One thread block owns a "pack" of rods (a consecutive run in CSR order, or rods listed by
// the best-fit packer, each with its offsets into the global arrays) and stages their nodes,
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

#include <algorithm>

#include "rod_internal.h"
#include "rod_step_device.cuh"

namespace rod {

namespace {

// ------------------------------------------------------------------------- the pack kernel

// The work of one pack, shared by the block kernel (pack in shared memory, one block) and the
// cooperative kernel (pack in global memory, every block of the grid); stage_sync is the
// block's or the grid's barrier.  FS: the feature set compiled in (see stage_elements).
template <int MODE, int FS = kFeatAll>
__device__ __forceinline__ void pack_body(const StepParams& P, const Pack& pk, Smem& m, int64_t n_steps, double t0,
                                          double dt, int last_half, double* acc_v, double* acc_w) {
  // a step after a latched error (non-finite state, contact overflow) is skipped: a block
  // decides once for all its threads; the blocks of a cooperative grid all read the word
  // before any of them can set it (after the last grid barrier)
  if (MODE == MODE_ONE_STEP) {
    const bool stop = *(volatile int*)P.err != 0;
    if (m.grid ? stop : __syncthreads_or(stop)) return;
  }
  const int Ep = pk.nelem, Np = pk.nnode;

  stage_pack(P, pk, m);


  if (MODE == MODE_KIN_HALF) {
    kinematic(P, pk, m, 0.5 * dt);
    stage_sync(m);
  } else if (MODE == MODE_RHS) {
    actuation_values(P, pk, m, t0);
    stage_elements(P, pk, m);
    stage_sync(m);
    stage_voronoi(P, pk, m);
    stage_sync(m);
    stage_rotation<MODE_RHS>(P, pk, m, dt, 0.0, acc_w);
    stage_translation<MODE_RHS>(P, pk, m, dt, acc_v, t0);
    return;
  } else {
    if (MODE == MODE_STEPS) {
      kinematic(P, pk, m, 0.5 * dt);
      stage_sync(m);
    }
    const double tbase = P.t_dev ? *P.t_dev : t0;
    const bool timed = has_time_values(P);
    if (n_steps > 0) actuation_values(P, pk, m, tbase + 0.5 * dt);
    for (int64_t s = 0; s < n_steps; ++s) {
      stage_elements<FS>(P, pk, m);
      stage_sync(m);
      stage_voronoi<FS>(P, pk, m);
      stage_sync(m);
      // rate updates fused with the following kinematic stage: each thread moves only the
      // elements and nodes whose rates it has just updated
      const bool last = (s == n_steps - 1);
      const double h = (last && (MODE == MODE_STEPS || last_half)) ? 0.5 * dt : dt;
      const double t = tbase + (static_cast<double>(s) + 0.5) * dt;
      stage_rotation<MODE_STEPS, FS>(P, pk, m, dt, h, nullptr);
      stage_translation<MODE_STEPS, FS>(P, pk, m, dt, nullptr, t, h);
      // the next step's time values: their only readers (the element stage) are past a barrier;
      // the next step's element stage waits for the barrier below
      if (timed && !last) time_values(P, pk, m, t + dt);
      stage_sync(m);
    }
  }

  // ---- contact binning of the positions this launch leaves behind (the next step's
  // half-step positions): FP32 midpoint, half length and cell of every segment, counted per
  // cell with one atomic per distinct cell in the warp.
  const bool leaves_half = MODE == MODE_KIN_HALF || (MODE == MODE_ONE_STEP && !last_half);
  if (leaves_half && P.bin_count) {
    bool grid_bad = false, nonfinite = false;
    for (int i = m.t0; i < Ep; i += m.ts) {
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
      const int ge = i + m.dE[m.erod[i]];
      P.bin_cell[ge] = cell;
      P.bin_prox[ge] = make_float4(mid[0], mid[1], mid[2], 0.5f * len);
      const unsigned peers = __match_any_sync(__activemask(), cell);
      if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(P.bin_count + cell, __popc(peers));
    }
    if (nonfinite) atomicOr(P.err, ERR_NONFINITE);
    if (grid_bad) atomicOr(P.err, ERR_GRID);
  }

  // ---- write back.  Non-finite values are found from the largest exponent field on the
  // integer pipe (all ones: Inf or NaN), which leaves the FP64 pipe to the step's arithmetic.
  // With the skin list, every segment also gets its FP32 proxy (midpoint, half length, half
  // edge, radius) from the node positions the kinematic stage rounded to FP32 in shared memory
  // (or rounded here where the pack has no room for them).
  unsigned expo = 0u;
  const bool prox = leaves_half && P.seg_prox != nullptr;
  for (int i = m.t0; i < Ep; i += m.ts) {
    const int ge = i + m.dE[m.erod[i]];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      const double q = m.QQ[a * m.CE + i];
      expo = max(expo, exp_field(q));
      P.Q[a * P.E + ge] = q;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double ww = m.WW[c * m.CE + i];
      expo = max(expo, exp_field(ww));
      P.w[c * P.E + ge] = ww;
    }
    if (prox) {
      const int r = m.erod[i];
      const int j = i + r;
      float p0[3], p1[3], he[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        p0[c] = m.XF ? m.XF[c * m.CN + j] : static_cast<float>(m.X[c * m.CN + j]);
        p1[c] = m.XF ? m.XF[c * m.CN + j + 1] : static_cast<float>(m.X[c * m.CN + j + 1]);
        he[c] = 0.5f * (p1[c] - p0[c]);
      }
      const float hl = sqrtf(fmaf(he[0], he[0], fmaf(he[1], he[1], he[2] * he[2])));
      P.seg_prox[2 * static_cast<int64_t>(ge)] =
          make_float4(0.5f * (p0[0] + p1[0]), 0.5f * (p0[1] + p1[1]), 0.5f * (p0[2] + p1[2]), hl);
      P.seg_prox[2 * static_cast<int64_t>(ge) + 1] = make_float4(he[0], he[1], he[2], P.rods[m.grod[r]].radius_f);
    }
  }
  // Upper bound of the node displacement since the skin list's build, in FP32: with xf, rf the
  // FP32 roundings of the position and of the build's position (each within 2^-24 of its
  // magnitude), |x - x_ref| <= |xf - rf| + 2^-24 sum_c (|xf_c| + |rf_c|) (to first order);
  // the factor and the coefficient below cover that and the rounding of these expressions.
  const bool track = P.disp_ref != nullptr && MODE != MODE_RHS;
  float dmax = 0.f;
  for (int j = m.t0; j < Np; j += m.ts) {
    const int64_t gn = j + m.dN[m.nrod[j]];
    float s2 = 0.f, mag = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double xx = m.X[c * m.CN + j], vv = m.VN[c * m.CN + j];
      expo = max(expo, max(exp_field(xx), exp_field(vv)));
      P.x[c * P.N + gn] = xx;
      P.v[c * P.N + gn] = vv;
      if (track) {
        const float xf = m.XF ? m.XF[c * m.CN + j] : static_cast<float>(xx);
        const float rf = P.disp_ref[c * P.N + gn];
        const float d = xf - rf;
        s2 = fmaf(d, d, s2);
        mag += fabsf(xf) + fabsf(rf);
      }
    }
    if (track) dmax = fmaxf(dmax, fmaf(sqrtf(s2), 1.000001f, 1.25e-7f * mag));
  }
  if (track) {
    // warp maximum, then one atomic per warp whose maximum raises the word (non-negative
    // doubles order like their bit patterns; the square of an FP32 value is exact in FP64)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0) {
      const double d2 = static_cast<double>(dmax) * static_cast<double>(dmax);
      const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(d2));
      if (bits > *(volatile unsigned long long*)P.disp_word) atomicMax(P.disp_word, bits);
    }
  }
  const bool bad = expo == kExpAllOnes;
  if (m.grid) {
    if (__any_sync(__activemask(), bad) && (threadIdx.x & 31) == __ffs(__activemask()) - 1) atomicOr(P.err, ERR_NONFINITE);
  } else if (__syncthreads_or(bad) && threadIdx.x == 0) {
    atomicOr(P.err, ERR_NONFINITE);
  }
}

template <int MODE, int FS>
__device__ __forceinline__ void block_pack(const StepParams& P, const LaunchShape& S, int64_t n_steps, double t0,
                                           double dt, int last_half, double* acc_v, double* acc_w) {
  extern __shared__ double smem_d[];
  const Pack pk = P.packs[blockIdx.x];
  Smem m = carve(smem_d, S);
  if (P.xf_smem_off) m.XF = reinterpret_cast<float*>(reinterpret_cast<char*>(smem_d) + P.xf_smem_off);
  pack_body<MODE, FS>(P, pk, m, n_steps, t0, dt, last_half, acc_v, acc_w);
}

template <int MODE>
__global__ void __launch_bounds__(512) pack_kernel(StepParams P, LaunchShape S, int64_t n_steps,
                                                   double t0, double dt, int last_half, double* acc_v, double* acc_w) {
  block_pack<MODE, kFeatAll>(P, S, n_steps, t0, dt, last_half, acc_v, acc_w);
}

// The plain step, held to 80 registers a thread for one step (no spills) and 84 for the step
// loop (4 bytes spilled), so that three 256-thread blocks fit an SM by registers as they do by
// the shared memory of 256-element packs.
template <int MODE>
__global__ void __maxnreg__(MODE == MODE_STEPS ? 84 : 80) pack_kernel_plain(StepParams P, LaunchShape S, int64_t n_steps,
                                                  double t0, double dt, int last_half, double* acc_v, double* acc_w) {
  block_pack<MODE, 0>(P, S, n_steps, t0, dt, last_half, acc_v, acc_w);
}

// Driven rods (actuation couples, damping or drag, and nothing else of kFeatAll): the cilia
// carpet.
template <int MODE>
__global__ void __launch_bounds__(512) pack_kernel_driven(StepParams P, LaunchShape S, int64_t n_steps, double t0,
                                                          double dt, int last_half, double* acc_v, double* acc_w) {
  block_pack<MODE, kFeatAct | kFeatDamp>(P, S, n_steps, t0, dt, last_half, acc_v, acc_w);
}

// One pack too long for a block: its working arrays live in global memory (scratch, carved
// like the shared-memory layout with the pack's own capacities) and the whole grid of a
// cooperative launch shares it, with grid-wide barriers between the stages.
template <int MODE>
__global__ void __launch_bounds__(256) pack_kernel_grid(StepParams P, Pack pk, LaunchShape S, double* scratch,
                                                        int64_t n_steps, double t0, double dt, int last_half,
                                                        double* acc_v, double* acc_w) {
  Smem m = carve(scratch, S);
  m.t0 = blockIdx.x * blockDim.x + threadIdx.x;
  m.ts = gridDim.x * blockDim.x;
  m.grid = true;
  pack_body<MODE>(P, pk, m, n_steps, t0, dt, last_half, acc_v, acc_w);
}


}  // namespace

size_t step_smem_bytes(const LaunchShape& s) {
  const size_t CE = s.cap_elems, CR = s.cap_rods, CN = CE + CR, CV = CE;
  const size_t doubles = 3 * CN + 3 * CN + 9 * CE + 3 * CE + 3 * CE + 3 * CE + CE + CE + 3 * CV + 3 * CV + CR + 4;
  const size_t ints = CR + 1 + 4 * CR;
  const size_t shorts = CE + CN + CV;
  return doubles * sizeof(double) + ints * sizeof(int) + shorts * sizeof(short) + 16;
}

const char* kernel_class_name(int k) {
  static const char* names[K_NUM_CLASSES] = {"pack_steps", "pack_one_step", "kin_half", "rhs", "contact_bin",
                                             "contact_scan", "contact_scatter", "contact_sort", "contact_gather",
                                             "contact_node_forces", "contact_list_build", "contact_list_force",
                                             "misc"};
  return (k >= 0 && k < K_NUM_CLASSES) ? names[k] : "?";
}

namespace {

template <int MODE>
cudaError_t launch_grid_packs(const StepParams& P, int64_t n_steps, double t0, double dt, int last_half, double* acc_v,
                              double* acc_w, cudaStream_t st) {
  static int sms = 0, per_sm = 0;
  cudaError_t e;
  if (!sms) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pack_kernel_grid<MODE>, 256, 0)))
      return e;
    per_sm = per_sm > 0 ? per_sm : 1;
  }
  for (int k = 0; k < P.n_long; ++k) {
    Pack pk = P.long_packs_h[k];
    LaunchShape ls;
    ls.cap_elems = pk.nelem;
    ls.cap_rods = pk.nrods;
    ls.threads = 256;
    const int need = (std::max(pk.nelem, pk.nnode) + 255) / 256;
    const int blocks = std::max(1, std::min(need, sms * per_sm));
    StepParams Pc = P;
    double* scratch = P.long_scratch;
    void* args[] = {&Pc, &pk, &ls, &scratch, &n_steps, &t0, &dt, &last_half, &acc_v, &acc_w};
    if ((e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(pack_kernel_grid<MODE>), dim3(blocks), dim3(256), args, 0,
                                         st)))
      return e;
  }
  return cudaSuccess;
}

template <int MODE, int FS>
void launch_block_packs(const StepParams& P, const LaunchShape& s, dim3 grid, dim3 block, size_t smem, int64_t n_steps,
                        double t0, double dt, int last_half, double* acc_v, double* acc_w, cudaStream_t st) {
  if constexpr (FS == kFeatAll) {
    cudaFuncSetAttribute(pack_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pack_kernel<MODE><<<grid, block, smem, st>>>(P, s, n_steps, t0, dt, last_half, acc_v, acc_w);
  } else if constexpr (FS == 0) {
    cudaFuncSetAttribute(pack_kernel_plain<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pack_kernel_plain<MODE><<<grid, block, smem, st>>>(P, s, n_steps, t0, dt, last_half, acc_v, acc_w);
  } else {
    static_assert(FS == (kFeatAct | kFeatDamp), "no kernel for this feature set");
    cudaFuncSetAttribute(pack_kernel_driven<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    pack_kernel_driven<MODE><<<grid, block, smem, st>>>(P, s, n_steps, t0, dt, last_half, acc_v, acc_w);
  }
}

// The step's features (kFeat* bits) that some rod of the system uses.
int step_features(const StepParams& P) {
  int f = 0;
  if (P.rest_sigma || P.rest_kappa) f |= kFeatRest;
  if (P.elem_couple || P.magnet || P.arc0 || P.n_walls > 0 || P.has_tip) f |= kFeatExt;
  if (P.has_act) f |= kFeatAct;
  if (P.has_damp_lin || P.has_damp_rot) f |= kFeatDamp;
  return f;
}

// Launch the kernel of the smallest instantiated feature set that covers the system's.
template <int MODE>
void launch_feature_packs(const StepParams& P, const LaunchShape& s, dim3 grid, dim3 block, size_t smem,
                          int64_t n_steps, double t0, double dt, int last_half, double* acc_v, double* acc_w,
                          cudaStream_t st) {
  const int f = step_features(P);
  if (f == 0) {
    launch_block_packs<MODE, 0>(P, s, grid, block, smem, n_steps, t0, dt, last_half, acc_v, acc_w, st);
  } else if ((f & ~(kFeatAct | kFeatDamp)) == 0) {
    launch_block_packs<MODE, kFeatAct | kFeatDamp>(P, s, grid, block, smem, n_steps, t0, dt, last_half, acc_v, acc_w, st);
  } else {
    launch_block_packs<MODE, kFeatAll>(P, s, grid, block, smem, n_steps, t0, dt, last_half, acc_v, acc_w, st);
  }
}

}  // namespace

cudaError_t launch_pack_kernel(const StepParams& P0, const LaunchShape& s, int mode, int64_t n_steps, double t0,
                               double dt, int last_half, double* acc_v, double* acc_w, cudaStream_t st,
                               const LaunchHook& hook) {
  size_t smem = step_smem_bytes(s);
  StepParams P = P0;
  P.xf_smem_off = 0;
  // FP32 node positions for the skin list's segment proxies, behind the pack's arrays when the
  // block's shared memory has room (otherwise the epilogue rounds the FP64 positions itself)
  if (P.seg_prox && mode != MODE_RHS) {
    const size_t off = (smem + 15) & ~size_t(15);
    const size_t need = off + sizeof(float) * 3 * static_cast<size_t>(s.cap_elems + s.cap_rods);
    if (need <= kMaxBlockSmem) {
      P.xf_smem_off = static_cast<int32_t>(off);
      smem = need;
    }
  }
  const dim3 grid(P.n_packs), block(s.threads);
  const int cls = mode == MODE_STEPS ? K_PACK_STEPS : mode == MODE_ONE_STEP ? K_PACK_ONE_STEP
                : mode == MODE_KIN_HALF ? K_KIN_HALF : K_RHS;
  hook.before(cls, st);
  struct After {
    const LaunchHook& h; int c; cudaStream_t s;
    ~After() { h.after(c, s); }
  } after_guard{hook, cls, st};
  cudaError_t e = cudaSuccess;
  switch (mode) {
    case MODE_STEPS: {
      if (P.n_packs > 0)
        launch_feature_packs<MODE_STEPS>(P, s, grid, block, smem, n_steps, t0, dt, last_half, acc_v, acc_w, st);
      if (P.n_long) e = launch_grid_packs<MODE_STEPS>(P, n_steps, t0, dt, last_half, acc_v, acc_w, st);
      break;
    }
    case MODE_ONE_STEP: {
      if (P.n_packs > 0)
        launch_feature_packs<MODE_ONE_STEP>(P, s, grid, block, smem, n_steps, t0, dt, last_half, acc_v, acc_w, st);
      if (P.n_long) e = launch_grid_packs<MODE_ONE_STEP>(P, n_steps, t0, dt, last_half, acc_v, acc_w, st);
      break;
    }
    case MODE_KIN_HALF: {
      if (P.n_packs > 0)
        launch_block_packs<MODE_KIN_HALF, kFeatAll>(P, s, grid, block, smem, n_steps, t0, dt, last_half, acc_v, acc_w, st);
      if (P.n_long) e = launch_grid_packs<MODE_KIN_HALF>(P, n_steps, t0, dt, last_half, acc_v, acc_w, st);
      break;
    }
    case MODE_RHS: {
      if (P.n_packs > 0)
        launch_block_packs<MODE_RHS, kFeatAll>(P, s, grid, block, smem, n_steps, t0, dt, last_half, acc_v, acc_w, st);
      if (P.n_long) e = launch_grid_packs<MODE_RHS>(P, n_steps, t0, dt, last_half, acc_v, acc_w, st);
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace rod
