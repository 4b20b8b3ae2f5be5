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
#include <cstring>
#include <vector>

#include "rod_contact.h"
#include "rod_cull.h"

namespace rod {

namespace {

// Largest number of segments one cell may hold; a denser cell (a collapsed or escaped
// configuration) latches ERR_OVERFLOW instead of running a quadratic search.
constexpr int kCellCap = 512;
// Longest element the contact grid covers, in units of the longest element at grid set-up.
constexpr double kStretchAllowance = 2.0;

// Closest points of P(s) = p0 + s d1, R(u) = q0 + u d2 on [0,1]^2 (minimise |r + s d1 - u d2|^2,
// r = p0 - q0): free minimiser s = (b f - c e)/(a e - b^2) clamped, u = (b s + f)/e; a clamped u
// re-solves s.  Parallel segments start from s = 0.  Quotients are taken as products with
// correctly rounded reciprocals (one per denominator): an FP64 division costs about three
// reciprocals on this part.
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
    u = fmin(fmax(f * __drcp_rn(e), 0.0), 1.0);
    return;
  }
  const double c = d1[0] * r[0] + d1[1] * r[1] + d1[2] * r[2];
  if (e <= 0.0) {
    u = 0.0;
    s = fmin(fmax(-c * __drcp_rn(a), 0.0), 1.0);
    return;
  }
  const double b = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
  const double den = a * e - b * b;
  s = (den != 0.0) ? fmin(fmax((b * f - c * e) * __drcp_rn(den), 0.0), 1.0) : 0.0;
  u = (b * s + f) * __drcp_rn(e);
  if (u < 0.0) {
    u = 0.0;
    s = fmin(fmax(-c * __drcp_rn(a), 0.0), 1.0);
  } else if (u > 1.0) {
    u = 1.0;
    s = fmin(fmax((b - c) * __drcp_rn(a), 0.0), 1.0);
  }
}

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
  const double d2 = dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2];
  if (!(d2 > 0.0)) return out;
  const double id = rsqrt(d2);              // 1 / d
  const double d = d2 * id;
  const double delta = (rada + radb) - d;
  if (!(delta > 0.0)) return out;
  const double nrm[3] = {dvec[0] * id, dvec[1] * id, dvec[2] * id};
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
    // 1 / max(|v_t|, v_slip) = min(1 / |v_t|, 1 / v_slip)
    const double sp2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
    const double fr = -A.mu * fmag * fmin(rsqrt(sp2), A.inv_vslip);
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

// Calls visit(b, rb) for every segment b of another rod in the 27-cell neighbourhood of slot q
// (cell-ordered records) that may come within r_a + r_b + extra of the slot's segment, in list
// order.  The three cells of each (y, z) row are consecutive in the list and scanned as one
// range; the next candidate's records are loaded while the current one is tested.
template <class Visit>
__device__ __forceinline__ void scan_neighbourhood(const ContactArgs& A, int64_t q, float extra, Visit& visit) {
  const float4 ga = A.recA[q];
  const int4 ba = A.recB[q];
  const float4 ea = A.recC[q];
  const int ra = ba.y;
  const float rada = __int_as_float(ba.z);
  const int cell = A.seg_cell[ba.x];
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
      int4 bb_next = make_int4(0, 0, 0, 0);
      float4 gb_next = make_float4(0.f, 0.f, 0.f, 0.f);
      if (b0 < b1) {
        bb_next = A.recB[b0];
        gb_next = A.recA[b0];
      }
      for (int t = b0; t < b1;) {
        const int tc = t;
        const int4 bb = bb_next;
        const float4 gb = gb_next;
        t = (bb.y == ra) ? bb.w : t + 1;  // own rod: skip its run in this cell
        if (t < b1) {
          bb_next = A.recB[t];
          gb_next = A.recA[t];
        }
        if (bb.y == ra) continue;
        if (!may_touch(ga, gb, ea, A.recC[tc], rada + __int_as_float(bb.z) + extra)) continue;
        visit(bb.x, bb.y);
      }
    }
  }
}

struct ForceSum {
  const ContactArgs& A;
  int a, ra;
  double fa[3], fb[3];
  __device__ ForceSum(const ContactArgs& args, int a_, int ra_) : A(args), a(a_), ra(ra_) {
#pragma unroll
    for (int c = 0; c < 3; ++c) fa[c] = fb[c] = 0.0;
  }
  __device__ void operator()(int b, int rb) {
    const PairForce pf = pair_force(A, a, ra, b, rb);
    if (pf.hit) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fa[c] += pf.fa[c];
        fb[c] += pf.fb[c];
      }
    }
  }
  __device__ void store(double* fseg, int64_t E) const {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      fseg[c * E + a] = fa[c];
      fseg[(3 + c) * E + a] = fb[c];
    }
  }
};

// The FP32 cull of segment a's skin list against the segment proxies of the current positions
// (written by the step kernel that produced them): the survivors as a bit mask over the list
// positions.  A segment whose list overflowed scans its neighbourhood of the last build with the
// skin bound instead (the build's records are stale by less than skin / 2 per node, which the
// skin covers), evaluating its pairs into f at once, and returns no survivors.
__device__ __forceinline__ unsigned cull_listed(const ContactArgs& A, int64_t a, ForceSum& f) {
  const int n = A.nbr_count[a];
  unsigned hit = 0u;
  if (n <= kNbrCap) {
    if (n > 0) {
      static_assert(kNbrCap <= 32, "the survivors of the cull are kept in a 32-bit mask");
      // groups of four: all indices, then all proxies, so that four independent loads are in flight
      const float4 ga = A.seg_prox[2 * a], ea = A.seg_prox[2 * a + 1];
      constexpr int kG = 4;
      for (int k0 = 0; k0 < n; k0 += kG) {
        int bs[kG];
        float4 gb[kG], eb[kG];
#pragma unroll
        for (int t = 0; t < kG; ++t) bs[t] = (k0 + t < n) ? A.nbr[(k0 + t) * A.E + a] : -1;
#pragma unroll
        for (int t = 0; t < kG; ++t) {
          if (bs[t] >= 0) {
            gb[t] = A.seg_prox[2 * (int64_t)bs[t]];
            eb[t] = A.seg_prox[2 * (int64_t)bs[t] + 1];
          }
        }
#pragma unroll
        for (int t = 0; t < kG; ++t)
          if (bs[t] >= 0 && may_touch(ga, gb[t], ea, eb[t], ea.w + eb[t].w)) hit |= 1u << (k0 + t);
      }
    }
  } else {
    scan_neighbourhood(A, A.slot_of[a], A.skin, f);
  }
  return hit;
}

constexpr int64_t kMaxCells = int64_t(1) << 24;
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;

// Order-preserving map of doubles to unsigned 64-bit keys (negative values reversed), so that
// atomicMin / atomicMax on the keys give the minimum / maximum of the doubles.
__device__ __forceinline__ unsigned long long okey(double v) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __forceinline__ double okey_decode(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  double v;
  std::memcpy(&v, &b, sizeof v);
  return v;
}

// Bounding box of the segment midpoints and the largest squared segment length (one block per
// rod, block reduction, one atomic per quantity); keys[7] is set when a midpoint or a length
// is not finite.
__global__ void bounds_kernel(const double* __restrict__ x, const RodConst* __restrict__ rods, int64_t N,
                              unsigned long long* keys) {
  const int r = blockIdx.x;
  const int64_t n0 = rods[r].node0;
  const int n = rods[r].n;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY}, l2 = 0.0;
  bool bad = false;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double ll = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double a = x[c * N + n0 + i], b = x[c * N + n0 + i + 1];
      const double m = 0.5 * (a + b);
      bad |= !isfinite(m);
      lo[c] = fmin(lo[c], m);
      hi[c] = fmax(hi[c], m);
      ll += (b - a) * (b - a);
    }
    bad |= !isfinite(ll);
    l2 = fmax(l2, ll);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      lo[c] = fmin(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
      hi[c] = fmax(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
    }
    l2 = fmax(l2, __shfl_xor_sync(0xffffffffu, l2, o));
  }
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      atomicMin(keys + c, okey(lo[c]));
      atomicMax(keys + 3 + c, okey(hi[c]));
    }
    atomicMax(keys + 6, okey(l2));
    if (bad) atomicOr(keys + 7, 1ull);
  }
}

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
  if (blockIdx.x == 0 && threadIdx.x == 0) *A.n_active = 0;  // refilled by list_active_kernel
  if (*(volatile int*)A.err != 0) return;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < A.E; q += (int64_t)gridDim.x * blockDim.x) {
    ListAppend l{A.nbr, A.E, A.recB[q].x, 0};
    scan_neighbourhood(A, q, A.skin, l);
    A.nbr_count[l.a] = l.n;
  }
}

// After a list build (gated): the segments with candidates, as a bit per segment index and as a
// compact list (warp-aggregated slots; the list's order does not matter, each segment's force
// is summed by one thread over its own candidates in list order).  Until the next build no
// other segment can touch anything, so the force kernel walks only these and the step kernels
// read only their forces.
__global__ void __launch_bounds__(256) list_active_kernel(ContactArgs A) {
  if (gated_off(A.gate)) return;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < A.E; base += stride) {
    const int64_t a = base + lane;
    const bool act = a < A.E && A.nbr_count[a] > 0;
    const unsigned mask = __ballot_sync(0xffffffffu, act);
    int slot = 0;
    if (lane == 0) {
      A.active_mask[base >> 5] = mask;
      if (mask) slot = atomicAdd(A.n_active, __popc(mask));
    }
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (act) A.active[slot + __popc(mask & ((1u << lane) - 1u))] = static_cast<int>(a);
  }
}

// Skin-list evaluation: the segments with candidates, one per lane of warps that stride over
// the active list.  Each lane culls its list in FP32 (cull_listed); the warp then packs the
// survivors of its 32 lanes, in lane and list order, into rounds of 32 and evaluates each round
// with one pair per lane (pair_force, FP64), passing the results back through shared memory;
// each lane adds the results of its own survivors in list order, so the sums are those of a
// lane that evaluated its survivors itself.  (Evaluated by their own lanes, a warp's survivors
// took as many FP64 passes as its busiest lane had survivors, with the other lanes masked --
// and a masked FP64 warp instruction costs the unit as much as a full one: 99.6 us per step in
// the packing's contact-dense window against 61 us packed.  One warp per segment, a lane per
// candidate, had measured 2.4x slower for the same reason.)  Two blocks per SM (128 registers,
// 108 bytes of spills around the out-of-line pair evaluation): 49 us; three (80 registers, 640
// bytes of spills): 61 us.
constexpr int kLfThreads = 256;
constexpr int kLfWarps = kLfThreads / 32;
__global__ void __launch_bounds__(kLfThreads, 2) list_force_kernel(ContactArgs A) {
  __shared__ int s_pair[kLfWarps][4][32];      // a, rod of a, b, rod of b of each slot of a round
  __shared__ double s_f[kLfWarps][6][32];      // the slot's contributions to a's two nodes
  __shared__ int s_hit[kLfWarps][32];
  if (*(volatile int*)A.err != 0) return;
  const int n = *A.n_active;
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int warps = gridDim.x * kLfWarps;
  for (int base = (blockIdx.x * kLfWarps + wb) * 32; base < n; base += warps * 32) {
    const int k = base + lane;
    const bool valid = k < n;
    const int a = valid ? A.active[k] : 0;
    const int ra = valid ? A.seg_rod[a] : 0;
    ForceSum f(A, a, ra);
    const unsigned hit = valid ? cull_listed(A, a, f) : 0u;
    // slots of this lane's survivors: [off, off + cnt) in the warp's order
    const int cnt = __popc(hit);
    int off = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, off, d);
      if (lane >= d) off += t;
    }
    const int total = __shfl_sync(0xffffffffu, off, 31);
    off -= cnt;
    for (int r0 = 0; r0 < total; r0 += 32) {
      // this lane's survivors that fall in the round's slots [r0, r0 + 32)
      if (off < r0 + 32 && off + cnt > r0) {
        unsigned h = hit;
        for (int idx = 0; h; ++idx) {
          const int kk = __ffs(h) - 1;
          h &= h - 1;
          const int slot = off + idx - r0;
          if (slot >= 0 && slot < 32) {
            const int b = A.nbr[kk * A.E + a];
            s_pair[wb][0][slot] = a;
            s_pair[wb][1][slot] = ra;
            s_pair[wb][2][slot] = b;
            s_pair[wb][3][slot] = A.seg_rod[b];
          }
        }
      }
      __syncwarp();
      if (r0 + lane < total) {
        const PairForce pf = pair_force(A, s_pair[wb][0][lane], s_pair[wb][1][lane], s_pair[wb][2][lane],
                                        s_pair[wb][3][lane]);
        s_hit[wb][lane] = pf.hit ? 1 : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          s_f[wb][c][lane] = pf.fa[c];
          s_f[wb][3 + c][lane] = pf.fb[c];
        }
      }
      __syncwarp();
      if (off < r0 + 32 && off + cnt > r0) {
        for (int idx = 0; idx < cnt; ++idx) {
          const int slot = off + idx - r0;
          if (slot >= 0 && slot < 32 && s_hit[wb][slot]) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              f.fa[c] += s_f[wb][c][slot];
              f.fb[c] += s_f[wb][3 + c][slot];
            }
          }
        }
      }
      __syncwarp();
    }
    if (valid) f.store(A.fseg, A.E);
  }
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

// Pair-set query: the visitor of one segment a records every pair (a, b), a < b, that survives
// the FP32 cull (a candidate) and, of those, every pair the FP64 evaluation finds in contact
// (positive overlap), in any order (atomic slots); counts keep rising past the capacity.
struct PairRecord {
  const ContactArgs& A;
  int a, ra;
  unsigned long long* counts;  // [0] pairs in contact, [1] candidates
  int64_t* out;
  int64_t cap;
  __device__ void operator()(int b, int rb) {
    if (b <= a) return;  // each pair once, from its lower segment
    atomicAdd(&counts[1], 1ull);
    if (!pair_force(A, a, ra, b, rb).hit) return;
    const unsigned long long k = atomicAdd(&counts[0], 1ull);
    if (k < static_cast<unsigned long long>(cap)) {
      out[2 * k] = a;
      out[2 * k + 1] = b;
    }
  }
};

__global__ void __launch_bounds__(256) pairs_kernel(ContactArgs A, unsigned long long* counts, int64_t* out,
                                                    int64_t cap) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= A.E) return;
  if (*(volatile int*)A.err != 0) return;
  const int4 ba = A.recB[q];
  PairRecord rec{A, ba.x, ba.y, counts, out, cap};
  scan_neighbourhood(A, q, 0.f, rec);
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
                  cs.nbr, cs.nbr_count, cs.slot_of, cs.x_ref, cs.seg_prox, cs.ctl, cs.bounds,
                  cs.active_mask, cs.active};
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
  cs.active_mask = nullptr;
  cs.active = nullptr;
  cs.ctl = nullptr;
  cs.bounds = nullptr;
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

namespace {
// Everything of a contact state that kernels captured in a graph take by value or by address.
std::vector<uint64_t> grid_signature(const ContactState& cs) {
  std::vector<uint64_t> v;
  auto d = [&v](double x) { uint64_t b; std::memcpy(&b, &x, sizeof b); v.push_back(b); };
  auto p = [&v](const void* q) { v.push_back(reinterpret_cast<uint64_t>(q)); };
  for (int c = 0; c < 3; ++c) {
    d(cs.lo[c]);
    v.push_back(static_cast<uint64_t>(cs.dim[c]));
  }
  d(cs.h); d(cs.inv_h); d(cs.l_allowed); d(cs.k); d(cs.c); d(cs.mu); d(cs.vslip); d(cs.skin);
  v.push_back(static_cast<uint64_t>(cs.ncell));
  v.push_back(static_cast<uint64_t>(cs.E));
  v.push_back(static_cast<uint64_t>(cs.N));
  v.push_back(static_cast<uint64_t>(cs.sm_count));
  const void* bufs[] = {cs.seg_rod, cs.seg_cell, cs.cell_count, cs.cell_start, cs.cell_fill, cs.block_sums,
                        cs.sorted, cs.prox, cs.recA, cs.recB, cs.recC, cs.fseg, cs.nbr, cs.nbr_count,
                        cs.slot_of, cs.x_ref, cs.seg_prox, cs.ctl, cs.active_mask, cs.active};
  for (const void* q : bufs) p(q);
  return v;
}
}  // namespace

rod_status contact_prepare(ContactState& cs, const std::vector<RodConst>& rods_h, const RodConst* rods_dev,
                           const double* x_dev, int64_t N, int64_t E, int R, cudaStream_t st, const LaunchHook& hook) {
  if (cs.grid_valid) return ROD_OK;
  if (cs.ctl && cs.ctl_live) {
    // the list state restarts below: keep the count of rebuilds run inside graphs so far
    cs.opened_before = contact_list_graph_rebuild_launches(cs, st) / kListRebuildKernels;
    cs.ctl_live = false;
  }
  // bounding box of the midpoints and the longest segment, reduced on the device
  cudaError_t e = cudaSuccess;
  if (!cs.bounds && (e = cudaMalloc(reinterpret_cast<void**>(&cs.bounds), 8 * sizeof(unsigned long long))))
    return cfail(ROD_ERR_CUDA, "contact grid: allocation", e);
  unsigned long long keys[8];
  for (int c = 0; c < 3; ++c) {
    keys[c] = ~0ull;      // minimum of the lower corner
    keys[3 + c] = 0ull;   // maximum of the upper corner
  }
  keys[6] = 0ull;
  keys[7] = 0ull;
  if ((e = cudaMemcpyAsync(cs.bounds, keys, sizeof keys, cudaMemcpyHostToDevice, st)))
    return cfail(ROD_ERR_CUDA, "contact grid: bounds", e);
  if (R > 0) {
    hook.before(K_MISC, st);
    bounds_kernel<<<R, 128, 0, st>>>(x_dev, rods_dev, N, cs.bounds);
    hook.after(K_MISC, st);
  }
  if ((e = cudaGetLastError()) || (e = cudaMemcpyAsync(keys, cs.bounds, sizeof keys, cudaMemcpyDeviceToHost, st)) ||
      (e = cudaStreamSynchronize(st)))
    return cfail(ROD_ERR_CUDA, "contact grid: bounds", e);
  if (keys[7] != 0ull) return cfail(ROD_ERR_NONFINITE, "contact grid: non-finite positions", cudaSuccess);
  double lo[3], hi[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = okey_decode(keys[c]);
    hi[c] = okey_decode(keys[3 + c]);
  }
  const double lmax = std::sqrt(okey_decode(keys[6]));
  double rmax = 0.0;
  for (int r = 0; r < R; ++r) rmax = std::max(rmax, rods_h[r].radius);
  for (int c = 0; c < 3; ++c)
    if (!std::isfinite(lo[c]) || !std::isfinite(hi[c]) || !std::isfinite(lmax))
      return cfail(ROD_ERR_NONFINITE, "contact grid: non-finite positions", cudaSuccess);
  // cell edge: a contacting pair's midpoints are closer than r_a + r_b + (l_a + l_b) / 2 (+ the
  // skin), so 2 r_max + l_max would do for the elements as they are now; the grid allows
  // elements up to twice the longest one at set-up (soft rods under stiff contact stretch
  // by tens of percent) before a longer one latches ROD_ERR_OVERFLOW
  const double skin = cs.skin > 0.0 ? cs.skin : 0.0;
  double h = std::max(cs.cell_size, 2.0 * rmax + kStretchAllowance * lmax + skin);
  if (!(h > 0.0)) h = 1.0;  // zero radii and lengths touch nothing: any positive edge is exact
  double ext[3], margin[3], dimd[3];
  double ncell_d = 0.0;
  // dimensions in double, clamped before the integer conversion (finite but huge extents of a
  // diverged state cannot overflow them); a larger cell edge keeps the search exact
  auto fit = [&](double hh) {
    ncell_d = 1.0;
    for (int c = 0; c < 3; ++c) {
      ext[c] = hi[c] - lo[c];
      margin[c] = std::max(0.1 * ext[c], 2.0 * hh);
      const double span = ext[c] + 2.0 * margin[c];
      dimd[c] = std::min(std::floor(span / hh) + 1.0, double(kMaxCells) + 1.0);
      ncell_d *= dimd[c];
    }
    return ncell_d <= double(kMaxCells);
  };
  bool fits = false;
  for (int iter = 0; iter < 64 && !(fits = fit(h)); ++iter) h *= 1.25;
  if (!fits) {
    // at most about 200 cells per dimension: span / h <= max(1.2 ext / h, ext / h + 4)
    h = std::max(h, 1.2 * std::max(ext[0], std::max(ext[1], ext[2])) / 200.0);
    fits = fit(h);
  }
  if (!fits) return cfail(ROD_ERR_OVERFLOW, "contact grid: the positions span too many cells", cudaSuccess);
  const int64_t ncell = static_cast<int64_t>(ncell_d);
  for (int c = 0; c < 3; ++c) {
    cs.dim[c] = static_cast<int>(dimd[c]);
    cs.lo[c] = lo[c] - margin[c];
  }
  cs.h = h;
  cs.inv_h = 1.0 / h;
  cs.ncell = ncell;
  // Cells are assigned from FP32 midpoints: a midpoint may move by a few ulps of the largest
  // coordinate, which the longest allowed element gives up (with a generous factor).
  double cmax = 0.0;
  for (int c = 0; c < 3; ++c) cmax = std::max(cmax, std::max(std::fabs(cs.lo[c]), std::fabs(cs.lo[c] + cs.dim[c] * h)));
  const double fp32_margin = 64.0 * 6e-8 * (1.0 + cmax);
  cs.l_allowed = h - 2.0 * rmax - skin - fp32_margin;
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
        (e = dev_alloc(&cs.ctl, 1)) || (e = dev_alloc(&cs.active_mask, (E + 31) / 32)) ||
        (e = dev_alloc(&cs.active, E)))
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
  // a new version (and with it a new capture of the contact step graph) only when something
  // the captured kernels read from their parameters has changed: the grid, the contact
  // constants or a buffer (a state set again with the same extent keeps the graph)
  const std::vector<uint64_t> sig = grid_signature(cs);
  if (sig != cs.signature) {
    cs.signature = sig;
    cs.version += 1;
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
  A.active_mask = cs.active_mask;
  A.active = cs.active;
  A.n_active = cs.ctl ? &cs.ctl->n_active : nullptr;
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

cudaError_t contact_pairs(ContactState& cs, const double* x, const double* v, const RodConst* rods, int64_t N,
                          int64_t E, int* err, unsigned long long* counts, int64_t* out, int64_t cap, cudaStream_t st,
                          const LaunchHook& hook) {
  cudaError_t e = enqueue_build(cs, x, rods, N, E, err, st, hook, false, nullptr);
  if (e) return e;
  if ((e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), st))) return e;
  const ContactArgs A = make_args(cs, x, v, rods, N, E, err, nullptr);
  hook.before(K_MISC, st);
  pairs_kernel<<<(E + 255) / 256, 256, 0, st>>>(A, counts, out, cap);
  hook.after(K_MISC, st);
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
  list_active_kernel<<<gb, 256, 0, st>>>(A);
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
  list_force_kernel<<<2 * std::max(cs.sm_count, 1), kLfThreads, 0, st>>>(A);
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
  P.fmask = cs.active_mask;
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
