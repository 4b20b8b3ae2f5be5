// rod_diag.cu -- energy and frame diagnostics of a state (rod_system_diagnostics).
//
// The energy of the discrete rod (Methods, the Cosserat model behind Eq. 1): translational
// kinetic energy of the nodes, rotational kinetic energy of the elements, shear/stretch energy
// of the element strains sigma = Q (x_{i+1} - x_i) / rl - d3 (frame components), bend/twist
// energy of the Voronoi curvatures kappa = -log(Q_{k+1} Q_k^T) / D, and the work potential of
// gravity and the constant tip forces; also the orthonormality of the directors and the tip
// positions.  One warp per rod; per-rod sums by warp shuffles, the totals by one block in a
// fixed order (the same bits on every call).  Not on the step path.
#include <cuda_runtime.h>

#include <cstdint>

#include "rod_diag.h"
#include "rod_step_device.cuh"

namespace rod {
namespace {

__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

__device__ __forceinline__ double warp_max(double a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
  return a;
}

__global__ void __launch_bounds__(256) diag_rod_kernel(DiagArgs A) {
  const int lane = threadIdx.x & 31;
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= A.R) return;  // whole warps leave together
  const RodConst* rc = A.rods + r;
  const int n = rc->n;
  const int64_t node0 = rc->node0, elem0 = rc->elem0, vor0 = rc->elem0 - r;
  const int64_t N = A.N, E = A.E, V = A.V;
  double kt = 0.0, kr = 0.0, es = 0.0, eb = 0.0, pot = 0.0, orth = 0.0;

  // nodes: 1/2 m |v|^2, -m g.x, and -F.x at the tip
  for (int j = lane; j <= n; j += 32) {
    const int64_t g = node0 + j;
    const double m = 1.0 / A.inv_m[g];
    const double x0 = A.x[g], x1 = A.x[N + g], x2 = A.x[2 * N + g];
    const double v0 = A.v[g], v1 = A.v[N + g], v2 = A.v[2 * N + g];
    kt += 0.5 * m * (v0 * v0 + v1 * v1 + v2 * v2);
    pot -= m * (A.gravity[0] * x0 + A.gravity[1] * x1 + A.gravity[2] * x2);
    if (j == n) {
      pot -= rc->tip[0] * x0 + rc->tip[1] * x1 + rc->tip[2] * x2;
      // the tip position, written by the lane that holds the last node
      A.per_rod[6 * A.R + r] = x0;
      A.per_rod[7 * A.R + r] = x1;
      A.per_rod[8 * A.R + r] = x2;
    }
  }
  // elements: 1/2 rho I_c rl w_c^2, 1/2 rl S_c (sigma_c - sigma0_c)^2, |Q Q^T - I|
  for (int i = lane; i < n; i += 32) {
    const int64_t ge = elem0 + i, gn = node0 + i;
    const double rl = A.rest_len[ge];
    double q[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) q[a] = A.Q[a * E + ge];
    const double l0 = A.x[gn + 1] - A.x[gn];
    const double l1 = A.x[N + gn + 1] - A.x[N + gn];
    const double l2 = A.x[2 * N + gn + 1] - A.x[2 * N + gn];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double wc = A.w[c * E + ge];
      kr += 0.5 * rc->rhoI[c] * rl * wc * wc;
      double s = (q[3 * c] * l0 + q[3 * c + 1] * l1 + q[3 * c + 2] * l2) / rl - (c == 2 ? 1.0 : 0.0);
      if (A.rest_sigma) s -= A.rest_sigma[c * E + ge];
      es += 0.5 * rl * rc->S[c] * s * s;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const double d = q[3 * a] * q[3 * b] + q[3 * a + 1] * q[3 * b + 1] + q[3 * a + 2] * q[3 * b + 2];
        orth = fmax(orth, fabs(d - (a == b ? 1.0 : 0.0)));
      }
  }
  // Voronoi points: 1/2 D B_c (kappa_c - kappa0_c)^2
  for (int k = lane; k < n - 1; k += 32) {
    const int64_t ge = elem0 + k, gv = vor0 + k;
    double qa[9], qb[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
      qa[a] = A.Q[a * E + ge];
      qb[a] = A.Q[a * E + ge + 1];
    }
    // R = Q_{k+1} Q_k^T, R_ab = d_a(k+1) . d_b(k); u = (R32 - R23, R13 - R31, R21 - R12) = 2 sin(t) n
    const double u0 = (qb[6] * qa[3] + qb[7] * qa[4] + qb[8] * qa[5]) - (qb[3] * qa[6] + qb[4] * qa[7] + qb[5] * qa[8]);
    const double u1 = (qb[0] * qa[6] + qb[1] * qa[7] + qb[2] * qa[8]) - (qb[6] * qa[0] + qb[7] * qa[1] + qb[8] * qa[2]);
    const double u2 = (qb[3] * qa[0] + qb[4] * qa[1] + qb[5] * qa[2]) - (qb[0] * qa[3] + qb[1] * qa[4] + qb[2] * qa[5]);
    const double f = theta_over_sin(u0 * u0 + u1 * u1 + u2 * u2, qa, qb);
    const double D = 0.5 * (A.rest_len[ge] + A.rest_len[ge + 1]);
    const double kf = -0.5 * f / D;
    const double kap[3] = {kf * u0, kf * u1, kf * u2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double kc = kap[c] - (A.rest_kappa ? A.rest_kappa[c * V + gv] : 0.0);
      eb += 0.5 * D * rc->B[c] * kc * kc;
    }
  }
  kt = warp_sum(kt);
  kr = warp_sum(kr);
  es = warp_sum(es);
  eb = warp_sum(eb);
  pot = warp_sum(pot);
  orth = warp_max(orth);
  if (lane == 0) {
    A.per_rod[r] = kt;
    A.per_rod[A.R + r] = kr;
    A.per_rod[2 * A.R + r] = es;
    A.per_rod[3 * A.R + r] = eb;
    A.per_rod[4 * A.R + r] = pot;
    A.per_rod[5 * A.R + r] = orth;
  }
}

// Totals over the rods: rows 0-4 summed, row 5 maximised; one block, fixed order.
__global__ void __launch_bounds__(256) diag_total_kernel(const double* per_rod, int R, double* totals) {
  __shared__ double red[8][6];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
#pragma unroll
    for (int c = 0; c < 5; ++c) acc[c] += per_rod[c * R + r];
    acc[5] = fmax(acc[5], per_rod[5 * R + r]);
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) acc[c] = warp_sum(acc[c]);
  acc[5] = warp_max(acc[5]);
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int c = 0; c < 6; ++c) red[wid][c] = acc[c];
  __syncthreads();
  if (threadIdx.x < 6) {
    const int c = threadIdx.x;
    double t = red[0][c];
    for (int k = 1; k < static_cast<int>(blockDim.x >> 5); ++k) t = (c < 5) ? t + red[k][c] : fmax(t, red[k][c]);
    totals[c] = t;
  }
}

}  // namespace

cudaError_t launch_diag_rows(const DiagArgs& A, cudaStream_t st) {
  if (A.R <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (static_cast<int64_t>(A.R) * 32 + threads - 1) / threads;
  diag_rod_kernel<<<static_cast<unsigned>(blocks), threads, 0, st>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_diag_totals(const double* per_rod, int R, double* totals_dev, cudaStream_t st) {
  diag_total_kernel<<<1, 256, 0, st>>>(per_rod, R, totals_dev);
  return cudaGetLastError();
}

}  // namespace rod
