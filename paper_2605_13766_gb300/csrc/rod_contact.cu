// rod_contact.cu -- rod-rod contact for sm_103a: uniform cell list (counting sort) and a
// gather-only segment-segment narrow phase.
//
// Broad phase (Results, "Fibrous granular materials": exhaustive search replaced by a hash
// grid, Fig. 2e): every segment's midpoint is binned into a uniform grid whose cell edge h is
// at least 2 r_max + l_max, so two segments in contact have midpoints in the same or adjacent
// cells.  Counting sort: count per cell, exclusive scan, scatter, then each cell's list is
// put in ascending segment order so that the force sums are reproducible.
//
// Narrow phase: each segment visits the 27 neighbour cells and, for every segment of another
// rod, (1) rejects it in FP32 when a lower bound of the segment distance, |m_a - m_b| minus
// the two half lengths, exceeds r_a + r_b by more than the FP32 rounding margin, then (2)
// evaluates the pair in FP64 exactly as the model defines it: closest points of the two
// segments (clamped two-parameter minimisation, lower segment index first so both members of
// the pair compute bit-identical values), overlap delta = r_a + r_b - d, force
// max(0, k delta - c v_rel . n) along n, split (1-s, s) onto the segment's nodes.  Each segment
// accumulates only its own share, so there are no atomics and no scatter conflicts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "rod_contact.h"

namespace rod {

namespace {

constexpr int64_t kMaxCells = int64_t(1) << 24;
// Largest number of segments one cell may hold; a denser cell (a collapsed or escaped
// configuration) latches ERR_OVERFLOW instead of running a quadratic search.
constexpr int kCellCap = 512;
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;

__global__ void seg_rod_kernel(const RodConst* rods, int R, int* seg_rod) {
  const int r = blockIdx.x;
  if (r >= R) return;
  const int e0 = rods[r].elem0, n = rods[r].n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) seg_rod[e0 + i] = r;
}

struct Grid {
  float lo[3];
  float inv_h;
  int dim[3];
  float l_allowed;
};

// Midpoint, half length and cell of every segment in FP32 (the cell only has to be consistent
// within one evaluation; the grid's slack covers the FP32 rounding of the midpoints), counted
// per cell with one atomic per distinct cell in the warp.
__global__ void bin_kernel(const double* __restrict__ x, const int* __restrict__ seg_rod, int64_t N, int64_t E, Grid g,
                           int* __restrict__ seg_cell, int* __restrict__ cell_count, float4* __restrict__ prox,
                           int* err) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= E) return;
  const int64_t j = a + seg_rod[a];
  float mid[3], ll = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float p0 = (float)x[c * N + j], p1 = (float)x[c * N + j + 1];
    mid[c] = 0.5f * (p0 + p1);
    ll = fmaf(p1 - p0, p1 - p0, ll);
  }
  const float len = sqrtf(ll);
  const bool finite = isfinite(mid[0]) && isfinite(mid[1]) && isfinite(mid[2]) && isfinite(len);
  if (!finite) atomicOr(err, ERR_NONFINITE);
  else if (!(len <= g.l_allowed)) atomicOr(err, ERR_GRID);
  int ic[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float f = floorf((mid[c] - g.lo[c]) * g.inv_h);
    f = fminf(fmaxf(f, 0.f), (float)(g.dim[c] - 1));  // NaN -> 0 via fmaxf
    ic[c] = (int)f;
  }
  const int cell = (ic[2] * g.dim[1] + ic[1]) * g.dim[0] + ic[0];
  seg_cell[a] = cell;
  // consecutive segments of a rod share cells: one atomic per distinct cell in the warp
  const unsigned peers = __match_any_sync(__activemask(), cell);
  if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cell_count + cell, __popc(peers));
  prox[a] = make_float4(mid[0], mid[1], mid[2], 0.5f * len);
}

// ---- exclusive scan of cell_count[0..n) into cell_start[0..n], cell_start[n] = total
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot, int& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int t = lane < nw ? warp_tot[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == nw - 1) warp_tot[32] = ti;
  }
  __syncthreads();
  total = warp_tot[32];
  const int r = warp_tot[wid] + incl - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_tiles_kernel(const int* __restrict__ in, int64_t n,
                                                                   int* __restrict__ out, int* __restrict__ tile_sums) {
  __shared__ int wt[33];
  const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanPerThread;
  int v[kScanPerThread];
  int s = 0;
#pragma unroll
  for (int q = 0; q < kScanPerThread; ++q) {
    v[q] = (base + q < n) ? in[base + q] : 0;
    s += v[q];
  }
  int total;
  int off = block_exclusive_scan(s, wt, total);
#pragma unroll
  for (int q = 0; q < kScanPerThread; ++q) {
    if (base + q < n) out[base + q] = off;
    off += v[q];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int* sums, int64_t nt, int* out_total_slot) {
  __shared__ int wt[33];
  int carry = 0;
  for (int64_t b = 0; b < nt; b += kScanThreads) {
    const int64_t i = b + threadIdx.x;
    const int v = i < nt ? sums[i] : 0;
    int total;
    const int ex = block_exclusive_scan(v, wt, total);
    if (i < nt) sums[i] = ex + carry;
    carry += total;
  }
  if (threadIdx.x == 0) *out_total_slot = carry;
}

__global__ void scan_add_kernel(int* out, int64_t n, const int* sums) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] += sums[i / kScanTile];
}

__global__ void scatter_kernel(const int* __restrict__ seg_cell, int64_t E, int* __restrict__ fill,
                               int* __restrict__ sorted) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= E) return;
  const int pos = atomicAdd(fill + seg_cell[a], 1);
  sorted[pos] = (int)a;
}

__global__ void sort_cells_kernel(const int* __restrict__ start, int64_t ncell, int* __restrict__ sorted, int* err) {
  const int64_t cidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (cidx >= ncell) return;
  const int b = start[cidx], e = start[cidx + 1];
  if (e - b > kCellCap) {
    atomicOr(err, ERR_OVERFLOW);
    return;
  }
  if (*(volatile int*)err != 0) return;
  for (int i = b + 1; i < e; ++i) {  // insertion sort; cells hold a handful of segments
    const int key = sorted[i];
    int j = i - 1;
    while (j >= b && sorted[j] > key) {
      sorted[j + 1] = sorted[j];
      --j;
    }
    sorted[j + 1] = key;
  }
}

// Closest points of P(s) = p0 + s d1, R(u) = q0 + u d2 on [0,1]^2 (minimise |r + s d1 - u d2|^2,
// r = p0 - q0): free minimiser s = (b f - c e)/(a e - b^2) clamped, u = (b s + f)/e; a clamped u
// re-solves s.  Parallel segments start from s = 0.
__device__ __forceinline__ void closest(const double* p0, const double* p1, const double* q0, const double* q1,
                                        double& s, double& u) {
  double d1[3], d2[3], r[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    d1[c] = p1[c] - p0[c];
    d2[c] = q1[c] - q0[c];
    r[c] = p0[c] - q0[c];
  }
  const double a = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2];
  const double e = d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2];
  const double f = d2[0] * r[0] + d2[1] * r[1] + d2[2] * r[2];
  if (a <= 0.0 && e <= 0.0) {
    s = 0.0;
    u = 0.0;
    return;
  }
  if (a <= 0.0) {
    s = 0.0;
    u = fmin(fmax(f / e, 0.0), 1.0);
    return;
  }
  const double c = d1[0] * r[0] + d1[1] * r[1] + d1[2] * r[2];
  if (e <= 0.0) {
    u = 0.0;
    s = fmin(fmax(-c / a, 0.0), 1.0);
    return;
  }
  const double b = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
  const double den = a * e - b * b;
  s = (den != 0.0) ? fmin(fmax((b * f - c * e) / den, 0.0), 1.0) : 0.0;
  u = (b * s + f) / e;
  if (u < 0.0) {
    u = 0.0;
    s = fmin(fmax(-c / a, 0.0), 1.0);
  } else if (u > 1.0) {
    u = 1.0;
    s = fmin(fmax((b - c) / a, 0.0), 1.0);
  }
}

// Per-slot records in cell order, so that the narrow phase reads each candidate with two
// contiguous 16-byte loads: (FP32 midpoint, FP32 half length) and (segment, rod, FP32 radius).
__global__ void records_kernel(const int* __restrict__ sorted, const int* __restrict__ seg_rod,
                               const float4* __restrict__ prox, const RodConst* __restrict__ rods, int64_t E,
                               float4* __restrict__ recA, int4* __restrict__ recB) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= E) return;
  const int a = sorted[q];
  const int r = seg_rod[a];
  recA[q] = prox[a];
  recB[q] = make_int4(a, r, __float_as_int((float)rods[r].radius), 0);
}

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
  const RodConst* rods;
  double* fseg;
  int* err;
  int64_t N, E;
  int dim[3];
  double k, c;
  double mu, vslip;
};

struct PairForce {
  double fa[3], fb[3];
  bool hit;
};

// FP64 evaluation of one candidate pair (a, b) in canonical order (lower index first); returns
// the contributions to the two nodes of segment a.  Kept out of line: it runs only for the
// few candidates that survive the FP32 cull, and the scan loop stays small.
__device__ __noinline__ PairForce pair_force(const ContactArgs& A, int a, int ra, int b, int rb) {
  PairForce out;
  out.hit = false;
  const double rada = A.rods[ra].radius, radb = A.rods[rb].radius;
  const bool first = a < b;
  const int64_t na = a + ra, nb = b + rb;
  const int64_t nP = first ? na : nb, nQ = first ? nb : na;
  double P0[3], P1[3], Q0[3], Q1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    P0[c] = A.x[c * A.N + nP];
    P1[c] = A.x[c * A.N + nP + 1];
    Q0[c] = A.x[c * A.N + nQ];
    Q1[c] = A.x[c * A.N + nQ + 1];
  }
  double s, u;
  closest(P0, P1, Q0, Q1, s, u);
  double dvec[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) dvec[c] = (P0[c] + s * (P1[c] - P0[c])) - (Q0[c] + u * (Q1[c] - Q0[c]));
  const double d = sqrt(dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2]);
  const double delta = (rada + radb) - d;
  if (!(delta > 0.0) || d == 0.0) return out;
  const double nrm[3] = {dvec[0] / d, dvec[1] / d, dvec[2] / d};
  double vrel = 0.0, vr[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double vp0 = A.v[c * A.N + nP], vp1 = A.v[c * A.N + nP + 1];
    const double vq0 = A.v[c * A.N + nQ], vq1 = A.v[c * A.N + nQ + 1];
    vr[c] = ((1.0 - s) * vp0 + s * vp1) - ((1.0 - u) * vq0 + u * vq1);
    vrel += vr[c] * nrm[c];
  }
  double fmag = A.k * delta - A.c * vrel;
  if (fmag < 0.0) fmag = 0.0;
  // friction: -mu fmag v_t / max(|v_t|, v_slip) with v_t the tangential relative velocity
  double ft[3] = {0.0, 0.0, 0.0};
  if (A.mu > 0.0 && fmag > 0.0) {
    double vt[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) vt[c] = vr[c] - vrel * nrm[c];
    const double sp = sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
    const double fr = -A.mu * fmag / fmax(sp, A.vslip);
#pragma unroll
    for (int c = 0; c < 3; ++c) ft[c] = fr * vt[c];
  }
  // force on the first segment of the pair is +(fmag n + ft), on the second the opposite
  const double wa = first ? (1.0 - s) : -(1.0 - u);
  const double wb = first ? s : -u;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double fc = fmag * nrm[c] + ft[c];
    out.fa[c] = wa * fc;
    out.fb[c] = wb * fc;
  }
  out.hit = true;
  return out;
}

// One thread per slot of the cell-ordered list: threads of a warp share cells and their
// neighbour rows, so candidate records come from L1.  The three cells of each (y, z) row of
// the 3x3x3 neighbourhood are consecutive in the list and scanned as one range.
__global__ void __launch_bounds__(256, 4) gather_kernel(ContactArgs A) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= A.E) return;
  if (*(volatile int*)A.err != 0) return;  // latched error: the step is abandoned
  const float4 ga = A.recA[q];
  const int4 ba = A.recB[q];
  const int a = ba.x, ra = ba.y;
  const float rada = __int_as_float(ba.z);
  const float ma_inf = fmaxf(fabsf(ga.x), fmaxf(fabsf(ga.y), fabsf(ga.z)));
  double fa[3] = {0, 0, 0}, fb[3] = {0, 0, 0};
  const int cell = A.seg_cell[a];
  const int cx = cell % A.dim[0], cy = (cell / A.dim[0]) % A.dim[1], cz = cell / (A.dim[0] * A.dim[1]);
  const int x0 = max(cx - 1, 0), x1 = min(cx + 1, A.dim[0] - 1);
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = cz + dz;
    if (z < 0 || z >= A.dim[2]) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = cy + dy;
      if (y < 0 || y >= A.dim[1]) continue;
      const int row = (z * A.dim[1] + y) * A.dim[0];
      const int b0 = A.cell_start[row + x0], b1 = A.cell_start[row + x1 + 1];
      if (b1 - b0 > 3 * kCellCap) {
        atomicOr(A.err, ERR_OVERFLOW);
        continue;
      }
      // the next candidate's records are loaded while the current one is tested
      int4 bb_next = make_int4(0, 0, 0, 0);
      float4 gb_next = make_float4(0.f, 0.f, 0.f, 0.f);
      if (b0 < b1) {
        bb_next = A.recB[b0];
        gb_next = A.recA[b0];
      }
      for (int t = b0; t < b1; ++t) {
        const int4 bb = bb_next;
        const float4 gb = gb_next;
        if (t + 1 < b1) {
          bb_next = A.recB[t + 1];
          gb_next = A.recA[t + 1];
        }
        if (bb.y == ra) continue;
        // FP32 lower bound of the segment distance, |m_a - m_b| - (h_a + h_b) > r_a + r_b + tol,
        // compared squared: |m_a - m_b|^2 > (r_a + r_b + tol + h_a + h_b)^2 (tol covers the
        // rounding of both forms)
        const float ddx = ga.x - gb.x, ddy = ga.y - gb.y, ddz = ga.z - gb.z;
        const float dm2 = ddx * ddx + ddy * ddy + ddz * ddz;
        const float mb_inf = fmaxf(fabsf(gb.x), fmaxf(fabsf(gb.y), fabsf(gb.z)));
        const float tol = 1e-6f + 4e-6f * (ma_inf + mb_inf + ga.w + gb.w);
        const float reach = rada + __int_as_float(bb.z) + tol + ga.w + gb.w;
        if (dm2 > reach * reach) continue;
        const PairForce pf = pair_force(A, a, ra, bb.x, bb.y);
        if (pf.hit) {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            fa[c] += pf.fa[c];
            fb[c] += pf.fb[c];
          }
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    A.fseg[c * A.E + a] = fa[c];
    A.fseg[(3 + c) * A.E + a] = fb[c];
  }
}

__global__ void node_forces_kernel(const double* __restrict__ fseg, const RodConst* __restrict__ rods, int R, int64_t N,
                                   int64_t E, double* __restrict__ f) {
  const int r = blockIdx.x;
  if (r >= R) return;
  const int e0 = rods[r].elem0, n = rods[r].n, n0 = rods[r].node0;
  for (int j = threadIdx.x; j <= n; j += blockDim.x) {
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      if (j < n) s += fseg[c * E + e0 + j];
      if (j > 0) s += fseg[(3 + c) * E + e0 + j - 1];
      f[c * N + n0 + j] = s;
    }
  }
}

template <typename T>
cudaError_t dev_alloc(T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

}  // namespace

void contact_release(ContactState& cs) {
  void* ptrs[] = {cs.seg_rod, cs.seg_cell, cs.cell_count, cs.cell_start, cs.cell_fill,
                  cs.block_sums, cs.sorted, cs.prox, cs.fseg, cs.recA, cs.recB};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  cs.seg_rod = cs.seg_cell = cs.cell_count = cs.cell_start = cs.cell_fill = cs.block_sums = cs.sorted = nullptr;
  cs.prox = nullptr;
  cs.fseg = nullptr;
  cs.recA = nullptr;
  cs.recB = nullptr;
  cs.cap_cells = 0;
  cs.E = 0;
  cs.grid_valid = false;
}

static rod_status cfail(rod_status st, const char* what, cudaError_t e) {
  return internal_fail(st, what, e == cudaSuccess ? "" : cudaGetErrorString(e));
}

rod_status contact_prepare(ContactState& cs, const std::vector<RodConst>& rods_h, const RodConst* rods_dev,
                           const double* x_dev, int64_t N, int64_t E, int R, cudaStream_t st, const LaunchHook& hook) {
  if (cs.grid_valid) return ROD_OK;
  std::vector<double> x(3 * N);
  cudaError_t e = cudaMemcpyAsync(x.data(), x_dev, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cfail(ROD_ERR_CUDA, "contact grid: reading positions", e);
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double lmax = 0.0, rmax = 0.0;
  for (int r = 0; r < R; ++r) {
    rmax = std::max(rmax, rods_h[r].radius);
    const int64_t n0 = rods_h[r].node0;
    for (int i = 0; i < rods_h[r].n; ++i) {
      double ll = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double a = x[c * N + n0 + i], b = x[c * N + n0 + i + 1];
        const double m = 0.5 * (a + b);
        lo[c] = std::min(lo[c], m);
        hi[c] = std::max(hi[c], m);
        ll += (b - a) * (b - a);
      }
      lmax = std::max(lmax, std::sqrt(ll));
    }
  }
  for (int c = 0; c < 3; ++c)
    if (!std::isfinite(lo[c]) || !std::isfinite(hi[c]))
      return cfail(ROD_ERR_NONFINITE, "contact grid: non-finite positions", cudaSuccess);
  double h = std::max(cs.cell_size, 2.0 * rmax + 1.25 * lmax);
  double ext[3], margin[3];
  int64_t ncell = 0;
  for (int iter = 0; iter < 64; ++iter) {
    ncell = 1;
    for (int c = 0; c < 3; ++c) {
      ext[c] = hi[c] - lo[c];
      margin[c] = std::max(0.1 * ext[c], 2.0 * h);
      const double span = ext[c] + 2.0 * margin[c];
      cs.dim[c] = static_cast<int>(std::floor(span / h)) + 1;
      ncell *= cs.dim[c];
    }
    if (ncell <= kMaxCells) break;
    h *= 1.25;
  }
  for (int c = 0; c < 3; ++c) cs.lo[c] = lo[c] - margin[c];
  cs.h = h;
  cs.inv_h = 1.0 / h;
  cs.ncell = ncell;
  // Cells are assigned from FP32 midpoints: a midpoint may move by a few ulps of the largest
  // coordinate, which the longest allowed element gives up (with a generous factor).
  double cmax = 0.0;
  for (int c = 0; c < 3; ++c) cmax = std::max(cmax, std::max(std::fabs(cs.lo[c]), std::fabs(cs.lo[c] + cs.dim[c] * h)));
  const double fp32_margin = 64.0 * 6e-8 * (1.0 + cmax);
  cs.l_allowed = h - 2.0 * rmax - fp32_margin;
  cs.version += 1;
  if (cs.E != E) {
    if ((e = dev_alloc(&cs.seg_rod, E)) || (e = dev_alloc(&cs.seg_cell, E)) || (e = dev_alloc(&cs.sorted, E)) ||
        (e = dev_alloc(&cs.prox, E)) || (e = dev_alloc(&cs.fseg, 6 * E)) || (e = dev_alloc(&cs.recA, E)) ||
        (e = dev_alloc(&cs.recB, E)))
      return cfail(ROD_ERR_CUDA, "contact: allocation", e);
    cs.E = E;
  }
  if (cs.cap_cells < ncell) {
    const int64_t nt = (ncell + 1 + kScanTile - 1) / kScanTile;
    if ((e = dev_alloc(&cs.cell_count, ncell + 1)) || (e = dev_alloc(&cs.cell_start, ncell + 1)) ||
        (e = dev_alloc(&cs.cell_fill, ncell + 1)) || (e = dev_alloc(&cs.block_sums, nt + 1)))
      return cfail(ROD_ERR_CUDA, "contact: grid allocation", e);
    cs.cap_cells = ncell;
    cs.n_block_sums = nt;
  }
  hook.before(K_MISC, st);
  seg_rod_kernel<<<R, 64, 0, st>>>(rods_dev, R, cs.seg_rod);
  hook.after(K_MISC, st);
  if ((e = cudaGetLastError())) return cfail(ROD_ERR_CUDA, "contact: segment map", e);
  cs.grid_valid = true;
  return ROD_OK;
}

void contact_bin_params(const ContactState& cs, StepParams& P) {
  P.bin_prox = cs.prox;
  P.bin_cell = cs.seg_cell;
  P.bin_count = cs.cell_count;
  for (int c = 0; c < 3; ++c) {
    P.bin_lo[c] = (float)cs.lo[c];
    P.bin_dim[c] = cs.dim[c];
  }
  P.bin_inv_h = (float)cs.inv_h;
  P.bin_l_allowed = (float)cs.l_allowed;
}

cudaError_t contact_clear_counts(const ContactState& cs, cudaStream_t st) {
  return cudaMemsetAsync(cs.cell_count, 0, (cs.ncell + 1) * sizeof(int), st);
}

cudaError_t contact_compute(ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                            int64_t E, int R, int* err, cudaStream_t st, const LaunchHook& hook, bool prebinned) {
  cudaError_t e;
  (void)R;
  const int64_t n1 = cs.ncell + 1;
  const int tb = 256;
  const int64_t eb = (E + tb - 1) / tb;
  if (!prebinned) {
    if ((e = contact_clear_counts(cs, st))) return e;
    Grid g;
    for (int c = 0; c < 3; ++c) {
      g.lo[c] = (float)cs.lo[c];
      g.dim[c] = cs.dim[c];
    }
    g.inv_h = (float)cs.inv_h;
    g.l_allowed = (float)cs.l_allowed;
    hook.before(K_CONTACT_BIN, st);
    bin_kernel<<<eb, tb, 0, st>>>(x, cs.seg_rod, N, E, g, cs.seg_cell, cs.cell_count, cs.prox, err);
    hook.after(K_CONTACT_BIN, st);
    if ((e = cudaGetLastError())) return e;
  }
  const int64_t nt = (n1 + kScanTile - 1) / kScanTile;
  hook.before(K_CONTACT_SCAN, st);
  scan_tiles_kernel<<<nt, kScanThreads, 0, st>>>(cs.cell_count, n1, cs.cell_start, cs.block_sums);
  hook.after(K_CONTACT_SCAN, st);
  hook.before(K_CONTACT_SCAN, st);
  scan_sums_kernel<<<1, kScanThreads, 0, st>>>(cs.block_sums, nt, cs.block_sums + nt);
  hook.after(K_CONTACT_SCAN, st);
  hook.before(K_CONTACT_SCAN, st);
  scan_add_kernel<<<(n1 + 255) / 256, 256, 0, st>>>(cs.cell_start, n1, cs.block_sums);
  hook.after(K_CONTACT_SCAN, st);
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(cs.cell_fill, cs.cell_start, cs.ncell * sizeof(int), cudaMemcpyDeviceToDevice, st)))
    return e;
  hook.before(K_CONTACT_SCATTER, st);
  scatter_kernel<<<eb, tb, 0, st>>>(cs.seg_cell, E, cs.cell_fill, cs.sorted);
  hook.after(K_CONTACT_SCATTER, st);
  hook.before(K_CONTACT_SORT, st);
  sort_cells_kernel<<<(cs.ncell + 255) / 256, 256, 0, st>>>(cs.cell_start, cs.ncell, cs.sorted, err);
  hook.after(K_CONTACT_SORT, st);
  if ((e = cudaGetLastError())) return e;
  hook.before(K_CONTACT_SORT, st);
  records_kernel<<<eb, tb, 0, st>>>(cs.sorted, cs.seg_rod, cs.prox, rods, E, cs.recA, cs.recB);
  hook.after(K_CONTACT_SORT, st);
  if ((e = cudaGetLastError())) return e;
  ContactArgs A;
  A.x = x;
  A.v = v;
  A.seg_rod = cs.seg_rod;
  A.seg_cell = cs.seg_cell;
  A.cell_start = cs.cell_start;
  A.sorted = cs.sorted;
  A.prox = cs.prox;
  A.recA = cs.recA;
  A.recB = cs.recB;
  A.rods = rods;
  A.fseg = cs.fseg;
  A.N = N;
  A.E = E;
  for (int c = 0; c < 3; ++c) A.dim[c] = cs.dim[c];
  A.k = cs.k;
  A.c = cs.c;
  A.mu = cs.mu;
  A.vslip = cs.vslip;
  A.err = err;
  hook.before(K_CONTACT_GATHER, st);
  gather_kernel<<<(E + 255) / 256, 256, 0, st>>>(A);
  hook.after(K_CONTACT_GATHER, st);
  return cudaGetLastError();
}

cudaError_t contact_node_forces(const ContactState& cs, const RodConst* rods, int64_t N, int64_t E, int R, double* f,
                                cudaStream_t st, const LaunchHook& hook) {
  hook.before(K_CONTACT_NODE_FORCES, st);
  node_forces_kernel<<<R, 64, 0, st>>>(cs.fseg, rods, R, N, E, f);
  hook.after(K_CONTACT_NODE_FORCES, st);
  return cudaGetLastError();
}

}  // namespace rod
