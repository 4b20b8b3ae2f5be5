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
// rod, (1) rejects it in FP32 when a lower bound of the segment distance exceeds r_a + r_b by
// more than the FP32 rounding margin -- first |m_a - m_b| minus the two half lengths, then the
// separating-axis bound along u = (m_a - m_b)/|m_a - m_b|, |m_a - m_b| - |e_a . u| - |e_b . u|
// (e = half edge vector: a segment projects onto u as m . u +- |e . u|) -- then (2) evaluates
// the pair in FP64 exactly as the model defines it: closest points of the two segments
// (clamped two-parameter minimisation, lower segment index first so both members of the pair
// compute bit-identical values), overlap delta = r_a + r_b - d, force max(0, k delta -
// c v_rel . n) along n, split (1-s, s) onto the segment's nodes.  Each segment accumulates only
// its own share, so there are no atomics and no scatter conflicts.
//
// Skin list (optional): the same search with the bound raised by a skin records, per segment,
// the candidates that may come within r_a + r_b + skin; the distance of two segments moves by
// at most the sum of their endpoints' displacements, so while no node has moved by skin / 2
// since the build, every touching pair is on the list and a step evaluates only the listed
// pairs.  The step kernels raise the largest displacement; the rebuild kernels run, gated on
// the device, when it reaches skin / 2, and return at once otherwise (no host round trip, so
// the steps stay in one CUDA graph).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "rod_contact.h"
#include "rod_contact_device.cuh"

namespace rod {

namespace {

constexpr int64_t kMaxCells = int64_t(1) << 24;
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
__device__ __forceinline__ void bin_one(const double* __restrict__ x, const int* __restrict__ seg_rod, int64_t N,
                                        const Grid& g, int* __restrict__ seg_cell, int* __restrict__ cell_count,
                                        float4* __restrict__ prox, int* err, int64_t a) {
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

// A gate (null: always) lets the skin list's rebuild kernels return at once unless a rebuild
// is due; gated launches use a grid of a few blocks per SM and stride over the items.
__device__ __forceinline__ bool gated_off(const int* gate) { return gate && *(volatile const int*)gate == 0; }

__global__ void bin_kernel(const double* __restrict__ x, const int* __restrict__ seg_rod, int64_t N, int64_t E, Grid g,
                           int* __restrict__ seg_cell, int* __restrict__ cell_count, float4* __restrict__ prox,
                           int* err, const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < E; a += (int64_t)gridDim.x * blockDim.x)
    bin_one(x, seg_rod, N, g, seg_cell, cell_count, prox, err, a);
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
                                                                   int* __restrict__ out, int* __restrict__ tile_sums,
                                                                   const int* gate) {
  __shared__ int wt[33];
  if (gated_off(gate)) return;
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const int64_t base = tile * kScanTile + threadIdx.x * kScanPerThread;
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
    if (threadIdx.x == 0) tile_sums[tile] = total;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(int* sums, int64_t nt, int* out_total_slot,
                                                                  const int* gate) {
  __shared__ int wt[33];
  if (gated_off(gate)) return;
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

__global__ void scan_add_kernel(int* out, int64_t n, const int* sums, const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] += sums[i / kScanTile];
}

// Scatter cursors from the cell starts; the counts are cleared for the next rebuild.
__global__ void fill_kernel(const int* __restrict__ start, int64_t ncell, int* __restrict__ fill,
                            int* __restrict__ count, const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
    fill[c] = start[c];
    count[c] = 0;
  }
}

__global__ void scatter_kernel(const int* __restrict__ seg_cell, int64_t E, int* __restrict__ fill,
                               int* __restrict__ sorted, const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < E; a += (int64_t)gridDim.x * blockDim.x) {
    const int pos = atomicAdd(fill + seg_cell[a], 1);
    sorted[pos] = (int)a;
  }
}

__global__ void sort_cells_kernel(const int* __restrict__ start, int64_t ncell, int* __restrict__ sorted, int* err,
                                  const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t cidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cidx < ncell;
       cidx += (int64_t)gridDim.x * blockDim.x) {
    const int b = start[cidx], e = start[cidx + 1];
    if (e - b > kCellCap) {
      atomicOr(err, ERR_OVERFLOW);
      continue;
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
}

// Per-slot records in cell order, so that the narrow phase reads each candidate with
// contiguous 16-byte loads: (FP32 midpoint, FP32 half length), (segment, rod, FP32 radius, end
// of the rod's run) and, for candidates that pass the first bound, (FP32 half edge).  A cell
// lists its segments by ascending index and a rod's segments have consecutive indices, so the
// segments of one rod in a cell form one run of slots; a scan that meets a segment of its own
// rod (never a contact pair) jumps to the run's end.
__global__ void records_kernel(const int* __restrict__ sorted, const int* __restrict__ seg_rod,
                               const int* __restrict__ seg_cell, const int* __restrict__ cell_start,
                               const float4* __restrict__ prox, const double* __restrict__ x, int64_t N,
                               const RodConst* __restrict__ rods, int64_t E, float4* __restrict__ recA,
                               int4* __restrict__ recB, float4* __restrict__ recC, int* __restrict__ slot_of,
                               const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < E; q += (int64_t)gridDim.x * blockDim.x) {
    const int a = sorted[q];
    const int r = seg_rod[a];
    const int cell_end = cell_start[seg_cell[a] + 1];
    const int rod_end = rods[r].elem0 + rods[r].n;
    int run_end = (int)q + 1;
    while (run_end < cell_end && sorted[run_end] < rod_end) ++run_end;
    const int64_t na = (int64_t)a + r;
    float e[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) e[c] = (float)(0.5 * (x[c * N + na + 1] - x[c * N + na]));
    recA[q] = prox[a];
    recB[q] = make_int4(a, r, __float_as_int((float)rods[r].radius), run_end);
    recC[q] = make_float4(e[0], e[1], e[2], 0.f);
    if (slot_of) slot_of[a] = (int)q;
  }
}

// Direct evaluation: one thread per slot of the cell-ordered list (threads of a warp share
// cells and their neighbour rows, so candidate records come from L1).
__global__ void __launch_bounds__(256, 4) gather_kernel(ContactArgs A) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= A.E) return;
  if (*(volatile int*)A.err != 0) return;  // latched error: the step is abandoned
  const int4 ba = A.recB[q];
  ForceSum f(A, ba.x, ba.y);
  scan_neighbourhood(A, q, 0.f, f);
  f.store(A.fseg, A.E);
}

struct ListAppend {
  int* nbr;
  int64_t E;
  int a, n;
  __device__ void operator()(int b, int) {
    if (n < kNbrCap) nbr[n * E + a] = b;
    ++n;
  }
};

// Skin-list build (gated): the same scan with the bound raised by the skin.
__global__ void __launch_bounds__(256) list_build_kernel(ContactArgs A) {
  if (gated_off(A.gate)) return;
  if (*(volatile int*)A.err != 0) return;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < A.E; q += (int64_t)gridDim.x * blockDim.x) {
    ListAppend l{A.nbr, A.E, A.recB[q].x, 0};
    scan_neighbourhood(A, q, A.skin, l);
    A.nbr_count[l.a] = l.n;
  }
}

// Skin-list evaluation: one thread per segment.  The kernel is bound by the latency of its
// gathers, so it asks for three resident blocks per SM (80 registers; the spills sit around the
// out-of-line pair evaluation, which runs for the few survivors of the cull).
__global__ void __launch_bounds__(256, 3) list_force_kernel(ContactArgs A) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= A.E) return;
  if (*(volatile int*)A.err != 0) return;
  ForceSum f(A, (int)a, A.seg_rod[a]);
  listed_forces(A, a, f);
  f.store(A.fseg, A.E);
}

// Rebuild decision of this evaluation: requested, or a node has moved by skin / 2 (or the
// displacement is not finite).  Inside a graph it also opens or skips the conditional node
// that holds the rebuild kernels.
__global__ void list_decide_kernel(ListCtl* ctl, double limit2, cudaGraphConditionalHandle cond, int use_cond) {
  const double d2 = __longlong_as_double(static_cast<long long>(ctl->disp2));
  const int gate = (ctl->force != 0 || !(d2 < limit2)) ? 1 : 0;
  ctl->gate = gate;
  if (use_cond) {
    cudaGraphSetConditional(cond, static_cast<unsigned>(gate));
    ctl->opened += gate;
  }
}

// After a rebuild: the build's positions become the reference, the displacement restarts.
__global__ void list_snapshot_kernel(const double* __restrict__ x, int64_t n, float* __restrict__ x_ref, ListCtl* ctl,
                                     const int* gate) {
  if (gated_off(gate)) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x_ref[i] = static_cast<float>(x[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->disp2 = 0ull;
    ctl->force = 0;
    ctl->builds += 1;
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
                  cs.block_sums, cs.sorted, cs.prox, cs.fseg, cs.recA, cs.recB, cs.recC,
                  cs.nbr, cs.nbr_count, cs.slot_of, cs.x_ref, cs.seg_prox, cs.ctl};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  cs.seg_rod = cs.seg_cell = cs.cell_count = cs.cell_start = cs.cell_fill = cs.block_sums = cs.sorted = nullptr;
  cs.prox = nullptr;
  cs.fseg = nullptr;
  cs.recA = nullptr;
  cs.recB = nullptr;
  cs.recC = nullptr;
  cs.nbr = cs.nbr_count = cs.slot_of = nullptr;
  cs.x_ref = nullptr;
  cs.seg_prox = nullptr;
  cs.ctl = nullptr;
  cs.ctl_live = false;
  cs.N = 0;
  cs.cap_cells = 0;
  cs.E = 0;
  cs.grid_valid = false;
}

static rod_status cfail(rod_status st, const char* what, cudaError_t e) {
  return internal_fail(st, what, e == cudaSuccess ? "" : cudaGetErrorString(e));
}

int64_t contact_list_graph_rebuild_launches(const ContactState& cs, cudaStream_t st) {
  int64_t opened = cs.opened_before;
  if (cs.ctl && cs.ctl_live) {
    ListCtl c{};
    if (cudaMemcpyAsync(&c, cs.ctl, sizeof(ListCtl), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
        cudaStreamSynchronize(st) == cudaSuccess)
      opened += c.opened;
    cudaGetLastError();
  }
  return opened * kListRebuildKernels;
}

rod_status contact_prepare(ContactState& cs, const std::vector<RodConst>& rods_h, const RodConst* rods_dev,
                           const double* x_dev, int64_t N, int64_t E, int R, cudaStream_t st, const LaunchHook& hook) {
  if (cs.grid_valid) return ROD_OK;
  if (cs.ctl && cs.ctl_live) {
    // the list state restarts below: keep the count of rebuilds run inside graphs so far
    cs.opened_before = contact_list_graph_rebuild_launches(cs, st) / kListRebuildKernels;
    cs.ctl_live = false;
  }
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
  const double skin = cs.skin > 0.0 ? cs.skin : 0.0;
  double h = std::max(cs.cell_size, 2.0 * rmax + 1.25 * lmax + skin);
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
  cs.l_allowed = h - 2.0 * rmax - skin - fp32_margin;
  cs.version += 1;
  if (cs.E != E) {
    if ((e = dev_alloc(&cs.seg_rod, E)) || (e = dev_alloc(&cs.seg_cell, E)) || (e = dev_alloc(&cs.sorted, E)) ||
        (e = dev_alloc(&cs.prox, E)) || (e = dev_alloc(&cs.fseg, 6 * E)) || (e = dev_alloc(&cs.recA, E)) ||
        (e = dev_alloc(&cs.recB, E)) || (e = dev_alloc(&cs.recC, E)))
      return cfail(ROD_ERR_CUDA, "contact: allocation", e);
    cs.E = E;
    cs.N = 0;  // list buffers follow
  }
  if (skin > 0.0 && cs.N != N) {
    if ((e = dev_alloc(&cs.nbr, int64_t(kNbrCap) * E)) || (e = dev_alloc(&cs.nbr_count, E)) ||
        (e = dev_alloc(&cs.slot_of, E)) || (e = dev_alloc(&cs.x_ref, 3 * N)) || (e = dev_alloc(&cs.seg_prox, 2 * E)) ||
        (e = dev_alloc(&cs.ctl, 1)))
      return cfail(ROD_ERR_CUDA, "contact: skin list allocation", e);
    cs.N = N;
  }
  if (cs.sm_count == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      cs.sm_count = sms;
    cudaGetLastError();
    if (cs.sm_count <= 0) cs.sm_count = 1;
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
  // every structure starts empty; a skin list is rebuilt at its first evaluation
  if ((e = contact_clear_counts(cs, st))) return cfail(ROD_ERR_CUDA, "contact: clearing counts", e);
  if (skin > 0.0) {
    if ((e = cudaMemsetAsync(cs.ctl, 0, sizeof(ListCtl), st)) || (e = contact_list_invalidate(cs, st)))
      return cfail(ROD_ERR_CUDA, "contact: skin list reset", e);
    cs.ctl_live = true;
  }
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

namespace {

ContactArgs make_args(const ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                      int64_t E, int* err, const int* gate) {
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
  A.recC = cs.recC;
  A.gate = gate;
  A.nbr = cs.nbr;
  A.nbr_count = cs.nbr_count;
  A.slot_of = cs.slot_of;
  A.seg_prox = cs.seg_prox;
  A.skin = (float)cs.skin;
  A.rods = rods;
  A.fseg = cs.fseg;
  A.N = N;
  A.E = E;
  for (int c = 0; c < 3; ++c) A.dim[c] = cs.dim[c];
  A.k = cs.k;
  A.c = cs.c;
  A.mu = cs.mu;
  A.vslip = cs.vslip;
  A.inv_vslip = cs.vslip > 0.0 ? 1.0 / cs.vslip : INFINITY;
  A.err = err;
  return A;
}

// Cell structures and records of positions x: binning (unless the step kernel binned them),
// scan of the counts, scatter, per-cell sort, records.  Gated (skin list): every kernel returns
// at once unless the device gate is set, and strides over its items with a small grid.
cudaError_t enqueue_build(ContactState& cs, const double* x, const RodConst* rods, int64_t N, int64_t E, int* err,
                          cudaStream_t st, const LaunchHook& hook, bool prebinned, const int* gate) {
  cudaError_t e;
  const int64_t n1 = cs.ncell + 1;
  const int tb = 256;
  const int64_t cap = gate ? int64_t(8) * std::max(cs.sm_count, 1) : INT64_MAX;
  auto blocks = [&](int64_t n, int64_t per_block) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block, cap)));
  };
  if (!prebinned) {
    if (!gate && (e = contact_clear_counts(cs, st))) return e;
    Grid g;
    for (int c = 0; c < 3; ++c) {
      g.lo[c] = (float)cs.lo[c];
      g.dim[c] = cs.dim[c];
    }
    g.inv_h = (float)cs.inv_h;
    g.l_allowed = (float)cs.l_allowed;
    hook.before(K_CONTACT_BIN, st);
    bin_kernel<<<blocks(E, tb), tb, 0, st>>>(x, cs.seg_rod, N, E, g, cs.seg_cell, cs.cell_count, cs.prox, err, gate);
    hook.after(K_CONTACT_BIN, st);
    if ((e = cudaGetLastError())) return e;
  }
  const int64_t nt = (n1 + kScanTile - 1) / kScanTile;
  hook.before(K_CONTACT_SCAN, st);
  scan_tiles_kernel<<<blocks(nt, 1), kScanThreads, 0, st>>>(cs.cell_count, n1, cs.cell_start, cs.block_sums, gate);
  hook.after(K_CONTACT_SCAN, st);
  hook.before(K_CONTACT_SCAN, st);
  scan_sums_kernel<<<1, kScanThreads, 0, st>>>(cs.block_sums, nt, cs.block_sums + nt, gate);
  hook.after(K_CONTACT_SCAN, st);
  hook.before(K_CONTACT_SCAN, st);
  scan_add_kernel<<<blocks(n1, tb), tb, 0, st>>>(cs.cell_start, n1, cs.block_sums, gate);
  hook.after(K_CONTACT_SCAN, st);
  if ((e = cudaGetLastError())) return e;
  hook.before(K_CONTACT_SCATTER, st);
  fill_kernel<<<blocks(cs.ncell, tb), tb, 0, st>>>(cs.cell_start, cs.ncell, cs.cell_fill, cs.cell_count, gate);
  hook.after(K_CONTACT_SCATTER, st);
  hook.before(K_CONTACT_SCATTER, st);
  scatter_kernel<<<blocks(E, tb), tb, 0, st>>>(cs.seg_cell, E, cs.cell_fill, cs.sorted, gate);
  hook.after(K_CONTACT_SCATTER, st);
  hook.before(K_CONTACT_SORT, st);
  sort_cells_kernel<<<blocks(cs.ncell, tb), tb, 0, st>>>(cs.cell_start, cs.ncell, cs.sorted, err, gate);
  hook.after(K_CONTACT_SORT, st);
  if ((e = cudaGetLastError())) return e;
  hook.before(K_CONTACT_SORT, st);
  records_kernel<<<blocks(E, tb), tb, 0, st>>>(cs.sorted, cs.seg_rod, cs.seg_cell, cs.cell_start, cs.prox, x, N, rods,
                                              E, cs.recA, cs.recB, cs.recC, gate ? cs.slot_of : nullptr, gate);
  hook.after(K_CONTACT_SORT, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t contact_compute(ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                            int64_t E, int R, int* err, cudaStream_t st, const LaunchHook& hook, bool prebinned) {
  (void)R;
  cudaError_t e = enqueue_build(cs, x, rods, N, E, err, st, hook, prebinned, nullptr);
  if (e) return e;
  const ContactArgs A = make_args(cs, x, v, rods, N, E, err, nullptr);
  hook.before(K_CONTACT_GATHER, st);
  gather_kernel<<<(E + 255) / 256, 256, 0, st>>>(A);
  hook.after(K_CONTACT_GATHER, st);
  return cudaGetLastError();
}

cudaError_t contact_list_decide(ContactState& cs, cudaStream_t st, const LaunchHook& hook,
                                const cudaGraphConditionalHandle* cond) {
  const double half = 0.5 * cs.skin * (1.0 - 1e-6);
  hook.before(K_MISC, st);
  list_decide_kernel<<<1, 1, 0, st>>>(cs.ctl, half * half, cond ? *cond : cudaGraphConditionalHandle(0), cond ? 1 : 0);
  hook.after(K_MISC, st);
  return cudaGetLastError();
}

cudaError_t contact_list_rebuild(ContactState& cs, const double* x, const RodConst* rods, int64_t N, int64_t E,
                                 int* err, cudaStream_t st, const LaunchHook& hook) {
  const int* gate = &cs.ctl->gate;
  cudaError_t e = enqueue_build(cs, x, rods, N, E, err, st, hook, false, gate);
  if (e) return e;
  const ContactArgs A = make_args(cs, x, nullptr, rods, N, E, err, gate);
  const unsigned gb = static_cast<unsigned>(std::max(1, 8 * cs.sm_count));
  hook.before(K_CONTACT_LIST_BUILD, st);
  list_build_kernel<<<gb, 256, 0, st>>>(A);
  hook.after(K_CONTACT_LIST_BUILD, st);
  hook.before(K_CONTACT_LIST_BUILD, st);
  list_snapshot_kernel<<<gb, 256, 0, st>>>(x, 3 * N, cs.x_ref, cs.ctl, gate);
  hook.after(K_CONTACT_LIST_BUILD, st);
  return cudaGetLastError();
}

cudaError_t contact_list_force(ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                               int64_t E, int* err, cudaStream_t st, const LaunchHook& hook) {
  const ContactArgs A = make_args(cs, x, v, rods, N, E, err, &cs.ctl->gate);
  hook.before(K_CONTACT_LIST_FORCE, st);
  list_force_kernel<<<(E + 255) / 256, 256, 0, st>>>(A);
  hook.after(K_CONTACT_LIST_FORCE, st);
  return cudaGetLastError();
}

cudaError_t contact_list_compute(ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                                 int64_t E, int R, int* err, cudaStream_t st, const LaunchHook& hook) {
  (void)R;
  cudaError_t e = contact_list_decide(cs, st, hook, nullptr);
  if (e == cudaSuccess) e = contact_list_rebuild(cs, x, rods, N, E, err, st, hook);
  if (e == cudaSuccess) e = contact_list_force(cs, x, v, rods, N, E, err, st, hook);
  return e;
}

void contact_list_params(const ContactState& cs, StepParams& P) {
  P.disp_ref = cs.x_ref;
  P.disp_word = &cs.ctl->disp2;
  P.seg_prox = cs.seg_prox;
}

cudaError_t contact_list_invalidate(const ContactState& cs, cudaStream_t st) {
  if (!cs.ctl) return cudaSuccess;
  return cudaMemsetAsync(&cs.ctl->force, 0xff, sizeof(int), st);
}

cudaError_t contact_node_forces(const ContactState& cs, const RodConst* rods, int64_t N, int64_t E, int R, double* f,
                                cudaStream_t st, const LaunchHook& hook) {
  hook.before(K_CONTACT_NODE_FORCES, st);
  node_forces_kernel<<<R, 64, 0, st>>>(cs.fseg, rods, R, N, E, f);
  hook.after(K_CONTACT_NODE_FORCES, st);
  return cudaGetLastError();
}

}  // namespace rod
