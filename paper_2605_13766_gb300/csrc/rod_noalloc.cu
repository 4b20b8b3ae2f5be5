// rod_noalloc.cu -- rod-rod contact forces without any allocation (rod_contact_forces_noalloc).
//
// Some callers cannot allocate device memory at the moment they need contact forces: code
// that runs inside another framework's memory pool or allocator callback, real-time loops
// that must not touch the driver's allocator, or a process whose device memory is fully
// reserved by another runtime.  This entry point serves them: the caller passes its inputs
// and its output buffer, and every temporary (segment map, cell list, per-segment forces,
// grid bounds) lives in one file-scope __device__ array of fixed size.  It performs the same
// contact evaluation as the system's pipeline (uniform cell list over segment midpoints,
// FP32 conservative cull, FP64 closest-point spring-dashpot pair force split onto the segment
// nodes, forces gathered per segment without atomics), but builds the grid on the device from
// the current positions.
//
// The array is shared by every call on a device and keeps the last call's contents; the
// kernels below clear what must start at zero.  Calls that overlap on the GPU (two streams,
// or two host threads) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/rod.h"
#include "rod_contact.h"

namespace rod {
namespace noalloc {

constexpr int64_t kMaxSegs = ROD_NOALLOC_MAX_SEGMENTS;
constexpr int64_t kMaxCells = ROD_NOALLOC_MAX_CELLS;
constexpr int kCellCap = 512;
constexpr int kMaxDevices = 64;

struct GridState {
  unsigned long long lo_key[3];  // order-preserving keys of the midpoint bounds
  unsigned long long hi_key[3];
  unsigned long long lmax_key;   // longest segment
  unsigned long long rmax_key;   // largest radius
  double lo[3];
  double h, inv_h;
  int dim[3];
  int ncell;
  int err;
  int pad;
};

// section sizes (bytes), each rounded up to 256
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffSegRod = 0;
constexpr size_t kOffSegCell = kOffSegRod + align256(sizeof(int) * kMaxSegs);
constexpr size_t kOffSorted = kOffSegCell + align256(sizeof(int) * kMaxSegs);
constexpr size_t kOffProx = kOffSorted + align256(sizeof(int) * kMaxSegs);
constexpr size_t kOffFseg = kOffProx + align256(sizeof(float4) * kMaxSegs);
constexpr size_t kOffCount = kOffFseg + align256(sizeof(double) * 6 * kMaxSegs);
constexpr size_t kOffStart = kOffCount + align256(sizeof(int) * (kMaxCells + 1));
constexpr size_t kOffFill = kOffStart + align256(sizeof(int) * (kMaxCells + 1));
constexpr size_t kOffGrid = kOffFill + align256(sizeof(int) * kMaxCells);
constexpr size_t kScratchBytes = kOffGrid + align256(sizeof(GridState));

// The scratch.  In host code this name is only a host-side stand-in for the symbol; its device
// address comes from cudaGetSymbolAddress (scratch_on_current_device below).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct View {
  int* seg_rod;
  int* seg_cell;
  int* sorted;
  float4* prox;
  double* fseg;
  int* count;
  int* start;
  int* fill;
  GridState* grid;
};

__host__ __device__ inline View view_of(unsigned char* base) {
  View v;
  v.seg_rod = reinterpret_cast<int*>(base + kOffSegRod);
  v.seg_cell = reinterpret_cast<int*>(base + kOffSegCell);
  v.sorted = reinterpret_cast<int*>(base + kOffSorted);
  v.prox = reinterpret_cast<float4*>(base + kOffProx);
  v.fseg = reinterpret_cast<double*>(base + kOffFseg);
  v.count = reinterpret_cast<int*>(base + kOffCount);
  v.start = reinterpret_cast<int*>(base + kOffStart);
  v.fill = reinterpret_cast<int*>(base + kOffFill);
  v.grid = reinterpret_cast<GridState*>(base + kOffGrid);
  return v;
}

// order-preserving map of a double onto unsigned 64-bit integers (for atomicMin/atomicMax)
__device__ __forceinline__ unsigned long long okey(double d) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(d));
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ounkey(unsigned long long k) {
  const unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double(static_cast<long long>(u));
}

struct Args {
  const int* node_off;   // [R+1]
  const double* radius;  // [R]
  const double* x;
  const double* v;
  int64_t N, E;
  int R;
  double k, c, cell_size;
  double* f;
};

__device__ __forceinline__ int rod_of_segment(const int* node_off, int R, int a) {
  // largest r with node_off[r] - r <= a
  int lo = 0, hi = R - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (node_off[mid] - mid <= a) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void reset_kernel(View s) {
  const int t = threadIdx.x;
  if (t < 3) {
    s.grid->lo_key[t] = ~0ull;
    s.grid->hi_key[t] = 0ull;
  }
  if (t == 3) s.grid->lmax_key = 0ull;
  if (t == 4) s.grid->rmax_key = 0ull;
  if (t == 5) s.grid->err = 0;
}

__global__ void bounds_kernel(Args A, View s) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a < A.R) atomicMax(&s.grid->rmax_key, okey(A.radius[a]));
  if (a >= A.E) return;
  const int r = rod_of_segment(A.node_off, A.R, (int)a);
  s.seg_rod[a] = r;
  const int64_t j = a + r;
  double ll = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double p0 = A.x[c * A.N + j], p1 = A.x[c * A.N + j + 1];
    const double m = 0.5 * (p0 + p1);
    if (!isfinite(m)) atomicOr(&s.grid->err, ERR_NONFINITE);
    atomicMin(&s.grid->lo_key[c], okey(m));
    atomicMax(&s.grid->hi_key[c], okey(m));
    ll = fma(p1 - p0, p1 - p0, ll);
  }
  atomicMax(&s.grid->lmax_key, okey(sqrt(ll)));
}

__global__ void grid_kernel(Args A, View s) {
  GridState* g = s.grid;
  const double rmax = ounkey(g->rmax_key), lmax = ounkey(g->lmax_key);
  double h = fmax(A.cell_size, 2.0 * rmax + lmax);
  double lo[3], ext[3];
  for (int c = 0; c < 3; ++c) {
    lo[c] = ounkey(g->lo_key[c]);
    ext[c] = ounkey(g->hi_key[c]) - lo[c];
  }
  bool ok = isfinite(h);
  for (int c = 0; c < 3; ++c) ok = ok && isfinite(lo[c]) && isfinite(ext[c]);
  // zero radii and zero-length segments (h = 0) touch nothing: any positive cell edge is exact
  if (ok && !(h > 0.0)) h = 1.0;
  if (!ok) {
    g->err |= ERR_NONFINITE;
    for (int c = 0; c < 3; ++c) g->dim[c] = 1;
    g->ncell = 1;
    g->h = 1.0;
    g->inv_h = 1.0;
    return;
  }
  // Grow the cell edge until the grid fits the scratch (a larger edge keeps the search exact).
  // Dimensions are formed in double and clamped before any integer conversion, so extents of
  // any finite size (a diverged state) cannot overflow them; when 200 growth steps are not
  // enough, the edge jumps to the largest extent / 63, which gives at most 64^3 cells.
  double dim[3], n = 0.0;
  auto fit = [&](double hh) {
    n = 1.0;
    for (int c = 0; c < 3; ++c) {
      dim[c] = fmin(floor(ext[c] / hh) + 1.0, (double)kMaxCells + 1.0);
      n *= dim[c];
    }
    return n <= (double)kMaxCells;
  };
  bool fits = false;
  for (int it = 0; it < 200 && !(fits = fit(h)); ++it) h *= 1.25;
  if (!fits) {
    h = fmax(h, fmax(ext[0], fmax(ext[1], ext[2])) / 63.0);
    fits = fit(h);
  }
  if (!fits) {  // unreachable for finite extents; kept so that no size is ever taken unchecked
    g->err |= ERR_OVERFLOW;
    for (int c = 0; c < 3; ++c) g->dim[c] = 1;
    g->ncell = 1;
    g->h = 1.0;
    g->inv_h = 1.0;
    return;
  }
  for (int c = 0; c < 3; ++c) {
    g->lo[c] = lo[c];
    g->dim[c] = static_cast<int>(dim[c]);
  }
  g->h = h;
  g->inv_h = 1.0 / h;
  g->ncell = static_cast<int>(n);
}

__global__ void clear_counts_kernel(View s) {
  const int n = s.grid->ncell + 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s.count[i] = 0;
}

__global__ void bin_kernel(Args A, View s) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= A.E) return;
  const GridState* g = s.grid;
  const int64_t j = a + s.seg_rod[a];
  double mid[3], ll = 0.0;
  for (int c = 0; c < 3; ++c) {
    const double p0 = A.x[c * A.N + j], p1 = A.x[c * A.N + j + 1];
    mid[c] = 0.5 * (p0 + p1);
    ll = fma(p1 - p0, p1 - p0, ll);
  }
  int ic[3];
  for (int c = 0; c < 3; ++c) {
    double q = floor((mid[c] - g->lo[c]) * g->inv_h);
    q = fmin(fmax(q, 0.0), (double)(g->dim[c] - 1));
    ic[c] = (int)q;
  }
  const int cell = (ic[2] * g->dim[1] + ic[1]) * g->dim[0] + ic[0];
  s.seg_cell[a] = cell;
  atomicAdd(s.count + cell, 1);
  s.prox[a] = make_float4((float)mid[0], (float)mid[1], (float)mid[2], (float)(0.5 * sqrt(ll)));
}

// one-block exclusive scan of count[0..ncell] into start[0..ncell]
__global__ void __launch_bounds__(1024) scan_kernel(View s) {
  __shared__ int part[1024];
  const int n = s.grid->ncell + 1;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * per, e = min(n, b + per);
  int sum = 0;
  for (int i = b; i < e; ++i) sum += s.count[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < blockDim.x; o <<= 1) {  // Hillis-Steele inclusive scan of the parts
    const int y = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += y;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int i = b; i < e; ++i) {
    s.start[i] = run;
    run += s.count[i];
  }
}

__global__ void fill_kernel(View s) {
  const int n = s.grid->ncell;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s.fill[i] = s.start[i];
}

__global__ void scatter_kernel(Args A, View s) {
  const int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a >= A.E) return;
  const int pos = atomicAdd(s.fill + s.seg_cell[a], 1);
  s.sorted[pos] = (int)a;
}

__global__ void sort_kernel(View s) {
  const int n = s.grid->ncell;
  for (int cidx = blockIdx.x * blockDim.x + threadIdx.x; cidx < n; cidx += gridDim.x * blockDim.x) {
    const int b = s.start[cidx], e = s.start[cidx + 1];
    if (e - b > kCellCap) {
      atomicOr(&s.grid->err, ERR_OVERFLOW);
      continue;
    }
    for (int i = b + 1; i < e; ++i) {
      const int key = s.sorted[i];
      int j = i - 1;
      while (j >= b && s.sorted[j] > key) {
        s.sorted[j + 1] = s.sorted[j];
        --j;
      }
      s.sorted[j + 1] = key;
    }
  }
}

// closest points of P(s) = p0 + s d1 and Q(u) = q0 + u d2 on [0,1]^2 (clamped minimisation)
__device__ __forceinline__ void closest_pts(const double* p0, const double* p1, const double* q0, const double* q1,
                                            double& s, double& u) {
  double d1[3], d2[3], r[3];
  for (int c = 0; c < 3; ++c) {
    d1[c] = p1[c] - p0[c];
    d2[c] = q1[c] - q0[c];
    r[c] = p0[c] - q0[c];
  }
  const double a = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2];
  const double e = d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2];
  const double f = d2[0] * r[0] + d2[1] * r[1] + d2[2] * r[2];
  if (a <= 0.0 && e <= 0.0) {
    s = u = 0.0;
    return;
  }
  if (a <= 0.0) {
    s = 0.0;
    u = fmin(fmax(f / e, 0.0), 1.0);
    return;
  }
  const double cc = d1[0] * r[0] + d1[1] * r[1] + d1[2] * r[2];
  if (e <= 0.0) {
    u = 0.0;
    s = fmin(fmax(-cc / a, 0.0), 1.0);
    return;
  }
  const double b = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
  const double den = a * e - b * b;
  s = (den != 0.0) ? fmin(fmax((b * f - cc * e) / den, 0.0), 1.0) : 0.0;
  u = (b * s + f) / e;
  if (u < 0.0) {
    u = 0.0;
    s = fmin(fmax(-cc / a, 0.0), 1.0);
  } else if (u > 1.0) {
    u = 1.0;
    s = fmin(fmax((b - cc) / a, 0.0), 1.0);
  }
}

__global__ void __launch_bounds__(128) gather_kernel(Args A, View s) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= A.E) return;
  const GridState* g = s.grid;
  const int a = s.sorted[q];
  double fa[3] = {0, 0, 0}, fb[3] = {0, 0, 0};
  if (g->err == 0) {
    const int ra = s.seg_rod[a];
    const double rada = A.radius[ra];
    const int64_t na = a + ra;
    const float4 pa = s.prox[a];
    const float ma_inf = fmaxf(fabsf(pa.x), fmaxf(fabsf(pa.y), fabsf(pa.z)));
    double xa0[3], xa1[3], va0[3], va1[3];
    for (int c = 0; c < 3; ++c) {
      xa0[c] = A.x[c * A.N + na];
      xa1[c] = A.x[c * A.N + na + 1];
      va0[c] = A.v[c * A.N + na];
      va1[c] = A.v[c * A.N + na + 1];
    }
    const int cell = s.seg_cell[a];
    const int cx = cell % g->dim[0], cy = (cell / g->dim[0]) % g->dim[1], cz = cell / (g->dim[0] * g->dim[1]);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int zz = cz + dz, yy = cy + dy, xx = cx + dx;
          if (zz < 0 || yy < 0 || xx < 0 || zz >= g->dim[2] || yy >= g->dim[1] || xx >= g->dim[0]) continue;
          const int cc = (zz * g->dim[1] + yy) * g->dim[0] + xx;
          const int b0 = s.start[cc], b1 = s.start[cc + 1];
          if (b1 - b0 > kCellCap) continue;  // flagged by sort_kernel
          for (int t = b0; t < b1; ++t) {
            const int b = s.sorted[t];
            const int rb = s.seg_rod[b];
            if (rb == ra) continue;
            const double radb = A.radius[rb];
            const float4 pb = s.prox[b];
            const float ddx = pa.x - pb.x, ddy = pa.y - pb.y, ddz = pa.z - pb.z;
            const float dm = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz);
            const float mb_inf = fmaxf(fabsf(pb.x), fmaxf(fabsf(pb.y), fabsf(pb.z)));
            const float tol = 1e-6f + 4e-6f * (ma_inf + mb_inf + pa.w + pb.w);
            if (dm - (pa.w + pb.w) > (float)rada + (float)radb + tol) continue;
            const bool first = a < b;
            const int64_t nb = b + rb;
            double P0[3], P1[3], Q0[3], Q1[3];
            for (int c = 0; c < 3; ++c) {
              const double xb0 = A.x[c * A.N + nb], xb1 = A.x[c * A.N + nb + 1];
              P0[c] = first ? xa0[c] : xb0;
              P1[c] = first ? xa1[c] : xb1;
              Q0[c] = first ? xb0 : xa0[c];
              Q1[c] = first ? xb1 : xa1[c];
            }
            double sp, up;
            closest_pts(P0, P1, Q0, Q1, sp, up);
            double dvec[3];
            for (int c = 0; c < 3; ++c) dvec[c] = (P0[c] + sp * (P1[c] - P0[c])) - (Q0[c] + up * (Q1[c] - Q0[c]));
            const double d = sqrt(dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2]);
            const double delta = (rada + radb) - d;
            if (!(delta > 0.0) || d == 0.0) continue;
            const double nrm[3] = {dvec[0] / d, dvec[1] / d, dvec[2] / d};
            double vrel = 0.0;
            for (int c = 0; c < 3; ++c) {
              const double vb0 = A.v[c * A.N + nb], vb1 = A.v[c * A.N + nb + 1];
              const double vp0 = first ? va0[c] : vb0, vp1 = first ? va1[c] : vb1;
              const double vq0 = first ? vb0 : va0[c], vq1 = first ? vb1 : va1[c];
              vrel += (((1.0 - sp) * vp0 + sp * vp1) - ((1.0 - up) * vq0 + up * vq1)) * nrm[c];
            }
            double fmag = A.k * delta - A.c * vrel;
            if (fmag < 0.0) fmag = 0.0;
            const double wa = first ? (1.0 - sp) : -(1.0 - up);
            const double wb = first ? sp : -up;
            for (int c = 0; c < 3; ++c) {
              fa[c] += wa * (fmag * nrm[c]);
              fb[c] += wb * (fmag * nrm[c]);
            }
          }
        }
  }
  for (int c = 0; c < 3; ++c) {
    s.fseg[c * A.E + a] = fa[c];
    s.fseg[(3 + c) * A.E + a] = fb[c];
  }
}

__global__ void node_forces_kernel(Args A, View s) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= A.N) return;
  // node j of rod r: left segment j - r - 1 (if j is not the rod's first node), right j - r
  int lo = 0, hi = A.R - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.node_off[mid] <= j) lo = mid; else hi = mid - 1;
  }
  const int r = lo;
  const bool hasR = j < A.node_off[r + 1] - 1, hasL = j > A.node_off[r];
  const int64_t seg = j - r;
  for (int c = 0; c < 3; ++c) {
    double sum = 0.0;
    if (hasR) sum += s.fseg[c * A.E + seg];
    if (hasL) sum += s.fseg[(3 + c) * A.E + seg - 1];
    A.f[c * A.N + j] = sum;
  }
}

std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
cudaError_t scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return cudaSuccess;
}

}  // namespace noalloc
}  // namespace rod

extern "C" rod_status rod_contact_forces_noalloc(int32_t n_rods, const int32_t* node_off, const double* radius,
                                                const double* x, const double* v, double k, double c,
                                                double cell_size, double* f, void* cuda_stream) {
  using namespace rod;
  using namespace rod::noalloc;
  if (n_rods <= 0 || !node_off || !radius || !x || !v || !f)
    return internal_fail(ROD_ERR_ARG, "rod_contact_forces_noalloc: null pointer or n_rods <= 0", "");
  if (!(k >= 0) || !(c >= 0) || !std::isfinite(k) || !std::isfinite(c) || !std::isfinite(cell_size))
    return internal_fail(ROD_ERR_ARG, "rod_contact_forces_noalloc: need finite k >= 0, c >= 0, cell_size", "");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // sizes: N = node_off[n_rods] is on the device; read it into a stack variable
  int32_t n_nodes = 0;
  cudaError_t e = cudaMemcpyAsync(&n_nodes, node_off + n_rods, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_contact_forces_noalloc: reading sizes", cudaGetErrorString(e));
  const int64_t N = n_nodes, E = (int64_t)n_nodes - n_rods;
  if (E < 1 || E < n_rods) return internal_fail(ROD_ERR_ARG, "rod_contact_forces_noalloc: bad node offsets", "");
  if (E > kMaxSegs) {
    char msg[160];
    snprintf(msg, sizeof msg, "%lld elements exceed the fixed scratch capacity of %lld", (long long)E,
             (long long)kMaxSegs);
    return internal_fail(ROD_ERR_OVERFLOW, "rod_contact_forces_noalloc", msg);
  }
  unsigned char* base = nullptr;
  e = scratch_on_current_device(&base);
  if (e != cudaSuccess)
    return internal_fail(ROD_ERR_CUDA, "rod_contact_forces_noalloc: cudaGetSymbolAddress", cudaGetErrorString(e));
  const View s = view_of(base);
  Args A;
  A.node_off = node_off;
  A.radius = radius;
  A.x = x;
  A.v = v;
  A.N = N;
  A.E = E;
  A.R = n_rods;
  A.k = k;
  A.c = c;
  A.cell_size = cell_size;
  A.f = f;
  const int tb = 256;
  const int eb = (int)((std::max<int64_t>(E, n_rods) + tb - 1) / tb);
  const int cells_blocks = (int)((kMaxCells + 1 + tb - 1) / tb);
  reset_kernel<<<1, 32, 0, st>>>(s);
  bounds_kernel<<<eb, tb, 0, st>>>(A, s);
  grid_kernel<<<1, 1, 0, st>>>(A, s);
  clear_counts_kernel<<<std::min(cells_blocks, 1024), tb, 0, st>>>(s);
  bin_kernel<<<(int)((E + tb - 1) / tb), tb, 0, st>>>(A, s);
  scan_kernel<<<1, 1024, 0, st>>>(s);
  fill_kernel<<<std::min(cells_blocks, 1024), tb, 0, st>>>(s);
  scatter_kernel<<<(int)((E + tb - 1) / tb), tb, 0, st>>>(A, s);
  sort_kernel<<<std::min(cells_blocks, 1024), tb, 0, st>>>(s);
  gather_kernel<<<(int)((E + 127) / 128), 128, 0, st>>>(A, s);
  node_forces_kernel<<<(int)((N + tb - 1) / tb), tb, 0, st>>>(A, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_contact_forces_noalloc: launch", cudaGetErrorString(e));
  int err = 0;
  e = cudaMemcpyAsync(&err, &s.grid->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_contact_forces_noalloc", cudaGetErrorString(e));
  if (err & ERR_NONFINITE) return internal_fail(ROD_ERR_NONFINITE, "rod_contact_forces_noalloc: non-finite positions", "");
  if (err & ERR_OVERFLOW)
    return internal_fail(ROD_ERR_OVERFLOW, "rod_contact_forces_noalloc: a cell holds more than 512 segments", "");
  return ROD_OK;
}
