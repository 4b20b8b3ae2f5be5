// rod_surrogate.cu -- learned per-rod surrogate of 50 fine steps (BF16 tensor cores, FP32
// accumulation, FP64 state update) with its own training kernels.
//
// Network (fixed): four 1D convolutions along a rod of 50 elements (51 node positions),
// kernel 5, zero padding, channels 32 (24 used) -> 64 -> 64 -> 64 -> 16 (15 used), SiLU
// between layers.  Input features per node position (raw_feature): position relative to the
// rod base, velocity, directors d1 and d2 and angular velocity of the element starting there,
// the relative rotation of the two elements meeting at that Voronoi point, the element's edge
// in its own frame (the last two carry the strains at a resolution BF16 keeps once shifted and
// scaled) and three samples of the base couple over the window.  Output: for the same 15
// state channels, the change over one window of fine steps minus a kinematic prior (x + T v,
// directors turned by the Rodrigues exponential of -T w), divided by per-channel scales.  The
// new state is prior + scale * output in FP64; the directors are re-orthonormalised
// (Gram-Schmidt on d1, d2; d3 = d1 x d2) and a clamp is re-applied.
//
// Inference (one persistent kernel per window call, tc_apply_kernel) runs the convolutions on
// the fifth-generation tensor cores (tcgen05: operands in shared memory, accumulator in tensor
// memory) and overlaps them with the FP64 features and update.  Training runs them kernel by
// kernel as implicit GEMMs on mma.sync.m16n8k16 (BF16 in, FP32 accumulate):
//   forward:  out[o, j] = b[o] + sum_{t,c} W[o, t, c] in[c, j + t - 2]    (M = C_out, N = j, K = 5 C_in)
//   input gradient: the same kernel with the tap-transposed weights and flipped taps
//   weight gradient: dW[o, t, c] = sum_{windows, j} g[o, j] in[c, j + t - 2]  (split over windows)
// Activations are stored [window][row][channel] with row = position + 2 (rows 0, 1 and
// 53..63 are the zero padding), so a pair of consecutive channels is one 32-bit load.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/rod.h"
#include "rod_contact.h"
#include "rod_fp.h"
#include "rod_tc.cuh"
#include "rod_internal.h"
#include "rod_rot.cuh"

namespace rod {
namespace sur {

constexpr int kPos = 51;     // node positions per rod
constexpr int kRows = 64;    // padded rows (position + 2)
constexpr int kTaps = 5;
constexpr int kC0 = 32;      // input channels (17 used)
constexpr int kC = 64;       // hidden channels
constexpr int kCO = 16;      // output channels (15 used)
constexpr int kFeat = 24;    // input features (see raw_feature)
constexpr int kOut = 15;

// parameter blocks (FP32 master copy): W1 [64][5*32], b1 [64], W2 [64][5*64], b2, W3, b3, W4 [16][5*64], b4 [16]
constexpr int kW1 = kC * kTaps * kC0, kW2 = kC * kTaps * kC, kW3 = kC * kTaps * kC, kW4 = kCO * kTaps * kC;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kW1, kOffW2 = kOffB1 + kC, kOffB2 = kOffW2 + kW2;
constexpr int kOffW3 = kOffB2 + kC, kOffB3 = kOffW3 + kW3, kOffW4 = kOffB3 + kC, kOffB4 = kOffW4 + kW4;
constexpr int kNumParams = kOffB4 + kCO;

// SiLU in FP32: the exponential and the quotient by their fast intrinsics (relative error below
// (4.5 + 1.2 |x|) 2^-23; -0 below x = -87.3, where the true value is under 1.5e-36 in size)
__device__ __forceinline__ float silu(float x) { return __fdividef(x, 1.0f + __expf(-x)); }
__device__ __forceinline__ float dsilu(float x) {
  const float s = 1.0f / (1.0f + __expf(-x));
  return s * (1.0f + x * (1.0f - s));
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return static_cast<uint32_t>(__bfloat16_as_ushort(lo)) | (static_cast<uint32_t>(__bfloat16_as_ushort(hi)) << 16);
}

__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

enum Epi : int { EPI_HIDDEN = 0, EPI_OUTPUT = 1, EPI_DGRAD = 2 };

// One thread block per window (rod); each warp takes (m-tile, n-tile) output tiles.
//   in   [B][64][CIN] BF16         W  [COUT][5*CIN] BF16 (tap-major K index k = t*CIN + c)
//   EPI_HIDDEN: out BF16 [B][64][COUT] = SiLU(acc + bias), pre FP32 [B][64][COUT] (optional)
//   EPI_OUTPUT: outf FP32 [B][51][COUT] = acc + bias
//   EPI_DGRAD:  out BF16 [B][64][COUT] = acc * SiLU'(pre_lo) (pre_lo: the lower layer's pre-activation)
template <int CIN, int COUT, int EPI, bool FLIP>
__global__ void __launch_bounds__(128) conv_kernel(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ W,
                                                   const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                   float* __restrict__ outf, float* __restrict__ pre,
                                                   const float* __restrict__ pre_lo, int nwin) {
  const int b = blockIdx.x;
  if (b >= nwin) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tg = lane & 3;
  constexpr int K = kTaps * CIN;
  constexpr int MT = COUT / 16, NT = 7;  // positions 0..55
  const __nv_bfloat16* inb = in + static_cast<int64_t>(b) * kRows * CIN;
  for (int tile = warp; tile < MT * NT; tile += 4) {
    const int m0 = (tile / NT) * 16, n0 = (tile % NT) * 8;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int j = n0 + g;  // this lane's B column (position)
#pragma unroll 4
    for (int kb = 0; kb < K / 16; ++kb) {
      const int t = (kb * 16) / CIN, cb = (kb * 16) % CIN;
      uint32_t af[4], bf[2];
      const __nv_bfloat16* wr0 = W + (m0 + g) * K + kb * 16 + 2 * tg;
      const __nv_bfloat16* wr1 = wr0 + 8 * K;
      af[0] = __ldg(reinterpret_cast<const unsigned int*>(wr0));
      af[1] = __ldg(reinterpret_cast<const unsigned int*>(wr1));
      af[2] = __ldg(reinterpret_cast<const unsigned int*>(wr0 + 8));
      af[3] = __ldg(reinterpret_cast<const unsigned int*>(wr1 + 8));
      const int row = FLIP ? (j - t + 4) : (j + t);
      const __nv_bfloat16* ir = inb + row * CIN + cb + 2 * tg;
      bf[0] = __ldg(reinterpret_cast<const unsigned int*>(ir));
      bf[1] = __ldg(reinterpret_cast<const unsigned int*>(ir + 8));
      mma_bf16(acc, af, bf);
    }
    // epilogue: acc[0] (o = m0+g, j = n0+2tg), acc[1] (o, j+1), acc[2] (o+8, j), acc[3] (o+8, j+1)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int o = m0 + g + ((q & 2) ? 8 : 0);
      const int jj = n0 + 2 * tg + (q & 1);
      float v = acc[q];
      if (EPI == EPI_OUTPUT) {
        if (jj < kPos) outf[(static_cast<int64_t>(b) * kPos + jj) * COUT + o] = v + bias[o];
      } else {
        const int64_t idx = (static_cast<int64_t>(b) * kRows + jj + 2) * COUT + o;
        float r = 0.f;
        if (jj < kPos) {
          if (EPI == EPI_HIDDEN) {
            v += bias[o];
            if (pre) pre[idx] = v;
            r = silu(v);
          } else {
            r = v * dsilu(pre_lo[idx]);
          }
        }
        out[idx] = __float2bfloat16_rn(r);
      }
    }
  }
}

// Partial weight gradient of one chunk of windows (grid.x), written without atomics:
//   part[chunk][o*K + t*CIN + c] = sum_{windows in chunk, j} g[b][j+2][o] in[b][j+t][c]
//   part[chunk][COUT*K + o]      = sum_{windows in chunk, j} g[b][j+2][o]
// grid.y: groups of 8 n-tiles (64 K columns); warp w owns m-tile w (COUT=64) or 0.  The chunks
// are summed in a fixed order by reduce_partials_kernel, so training is deterministic.
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) wgrad_kernel(const __nv_bfloat16* __restrict__ gout, const __nv_bfloat16* __restrict__ in,
                                                    float* __restrict__ part, int nwin, int win_per_block) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tg = lane & 3;
  constexpr int K = kTaps * CIN;
  constexpr int MT = COUT / 16;
  if (warp >= MT) return;
  const int m0 = warp * 16;
  const int nbase = blockIdx.y * 64;  // K columns handled by this block
  float acc[8][4];
#pragma unroll
  for (int s = 0; s < 8; ++s) acc[s][0] = acc[s][1] = acc[s][2] = acc[s][3] = 0.f;
  float bsum0 = 0.f, bsum1 = 0.f;
  const int w0 = blockIdx.x * win_per_block, w1 = min(nwin, w0 + win_per_block);
  for (int b = w0; b < w1; ++b) {
    const __nv_bfloat16* gb = gout + static_cast<int64_t>(b) * kRows * COUT;
    const __nv_bfloat16* ib = in + static_cast<int64_t>(b) * kRows * CIN;
    for (int jb = 0; jb < 64; jb += 16) {  // reduction over positions 0..63 (rows >= 53 are zero)
      // A(o, j) = g[j + 2][o]: rows m0+g (+8), cols jb + 2tg (+1), (+8)
      uint32_t af[4];
      auto gval = [&](int o, int jj) -> __nv_bfloat16 {
        return (jj + 2 < kRows) ? gb[(jj + 2) * COUT + o] : __float2bfloat16_rn(0.f);
      };
      af[0] = pack_bf16(gval(m0 + g, jb + 2 * tg), gval(m0 + g, jb + 2 * tg + 1));
      af[1] = pack_bf16(gval(m0 + g + 8, jb + 2 * tg), gval(m0 + g + 8, jb + 2 * tg + 1));
      af[2] = pack_bf16(gval(m0 + g, jb + 2 * tg + 8), gval(m0 + g, jb + 2 * tg + 9));
      af[3] = pack_bf16(gval(m0 + g + 8, jb + 2 * tg + 8), gval(m0 + g + 8, jb + 2 * tg + 9));
      if (blockIdx.y == 0) {
        for (int q = 0; q < 2; ++q) {
          const int jj = jb + 2 * tg + q;
          bsum0 += __bfloat162float(gval(m0 + g, jj)) + __bfloat162float(gval(m0 + g, jj + 8));
          bsum1 += __bfloat162float(gval(m0 + g + 8, jj)) + __bfloat162float(gval(m0 + g + 8, jj + 8));
        }
      }
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int ncol = nbase + s * 8 + g;  // K column = t*CIN + c
        if (ncol >= K) continue;
        const int t = ncol / CIN, c = ncol % CIN;
        // B(j, n) = in[j + t][c] for j = jb + 2tg (+1), (+8, +9)
        auto ival = [&](int jj) -> __nv_bfloat16 {
          const int row = jj + t;
          return row < kRows ? ib[row * CIN + c] : __float2bfloat16_rn(0.f);
        };
        uint32_t bf[2];
        bf[0] = pack_bf16(ival(jb + 2 * tg), ival(jb + 2 * tg + 1));
        bf[1] = pack_bf16(ival(jb + 2 * tg + 8), ival(jb + 2 * tg + 9));
        mma_bf16(acc[s], af, bf);
      }
    }
  }
  float* dW = part + static_cast<int64_t>(blockIdx.x) * (COUT * K + COUT);
  float* db = dW + COUT * K;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int nc = nbase + s * 8 + 2 * tg;
    if (nc >= K) continue;
    dW[(m0 + g) * K + nc] = acc[s][0];
    dW[(m0 + g) * K + nc + 1] = acc[s][1];
    dW[(m0 + g + 8) * K + nc] = acc[s][2];
    dW[(m0 + g + 8) * K + nc + 1] = acc[s][3];
  }
  if (blockIdx.y == 0) {
    // reduce the bias sums over the 4 lanes sharing a row
    for (int o = 1; o < 4; o <<= 1) {
      bsum0 += __shfl_xor_sync(0xffffffffu, bsum0, o);
      bsum1 += __shfl_xor_sync(0xffffffffu, bsum1, o);
    }
    if (tg == 0) {
      db[m0 + g] = bsum0;
      db[m0 + g + 8] = bsum1;
    }
  }
}

// grad[p] = sum over chunks c = 0, 1, ... of part[c][p], in that order
__global__ void reduce_partials_kernel(const float* __restrict__ part, int chunks, int n, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float acc = 0.f;
  for (int c = 0; c < chunks; ++c) acc += part[static_cast<int64_t>(c) * n + p];
  grad[p] = acc;
}

// ---- features, targets, loss, state update, Adam

struct WinState {          // a batch of rods of 50 elements in the system layout
  const double* x;         // [3][N]
  const double* v;
  const double* Q;         // [9][E], Q[(3a + k) E + e] = component k of director a
  const double* w;         // [3][E]
  int64_t N, E;
};

struct Scales {
  double in_shift[kFeat];  // raw feature shift (FP64: the raw features of raw_features_kernel)
  float in_shift_f[kFeat]; // the shift rounded to FP32: network input = (raw - shift) * scale in FP32
  float in_scale[kFeat];
  double out[kOut];        // state change = prior + out * network output
  double T;                // window length in time (window steps x dt)
  int prior_x;             // 1: positions have the prior x + T v (else x)
  int prior_q;             // 1: directors have the prior exp([-T w]x) Q (else Q)
  int keep_v;              // 1: velocities are v + output (residual), 0: output alone
  int keep_w;              // 1: angular velocities are w + output (residual), 0: output alone
};

// Directors d1, d2 (out[0..5]) of Q_new = exp([-T w]x) Q (rows: directors; d3 is not needed, the
// update rebuilds it from d1 x d2): the director update of a constant angular velocity w (local
// frame) held for the whole window, by the Rodrigues formula R = I + a K + b K^2 =
// (1 - b th^2) I + a K + b p p^T with p = -T w, K = [p]x, a = sin(th)/th, b = (1 - cos th)/th^2.
// No FP64 division: for th < 0.05 the Taylor polynomials of a and b in th^2 (the first omitted
// terms, th^8/9! and th^8/10!, are below 1e-16), otherwise sin and cos of th.
__device__ __forceinline__ void rotate_directors(const double w[3], double T, const double Q[9], double out[6]) {
  const double p0 = -T * w[0], p1 = -T * w[1], p2 = -T * w[2];
  const double th2 = fma(p0, p0, fma(p1, p1, p2 * p2));
  double a, b;
  rot_coeffs(th2, a, b);  // series cut per warp from its largest angle
  const double c0 = fma(-b, th2, 1.0);
  const double b0 = b * p0, b1 = b * p1;
  const double a0 = a * p0, a1 = a * p1, a2 = a * p2;
  const double R00 = fma(b0, p0, c0), R11 = fma(b1, p1, c0);
  const double R01 = fma(b0, p1, -a2), R10 = fma(b1, p0, a2);
  const double R02 = fma(b0, p2, a1), R12 = fma(b1, p2, -a0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double q0 = Q[k], q1 = Q[3 + k], q2 = Q[6 + k];
    out[k] = fma(R00, q0, fma(R01, q1, R02 * q2));
    out[3 + k] = fma(R10, q0, fma(R11, q1, R12 * q2));
  }
}

__device__ __forceinline__ void load_q(const double* Q, int64_t E, int64_t e, double q[9]) {
#pragma unroll
  for (int a = 0; a < 9; ++a) q[a] = Q[a * E + e];
}

// Raw feature c of window b at node position j; false where the feature is undefined.
//   0..2  node position minus the base node        3..5  node velocity
//   6..11 directors d1, d2 of element j            12..14 angular velocity of element j
//   15..17 half the axial vector of R - R^T, R = Q_j Q_{j-1}^T (relative rotation of the two
//          elements beside Voronoi point j; j = 1..49)
//   18..20 edge of element j in its own frame, Q_j (x_{j+1} - x_j)
//   21..23 base couple at the window's start, middle and end
__device__ bool raw_feature(const WinState& S, const double* __restrict__ act, int nwin, int b, int j, int c, double* out) {
  const int64_t node = static_cast<int64_t>(b) * kPos + j, node0 = static_cast<int64_t>(b) * kPos;
  const int64_t el = static_cast<int64_t>(b) * (kPos - 1) + j;
  const bool has_el = j < kPos - 1;
  if (c < 3) { *out = S.x[c * S.N + node] - S.x[c * S.N + node0]; return true; }
  if (c < 6) { *out = S.v[(c - 3) * S.N + node]; return true; }
  if (c < 12) { if (!has_el) return false; *out = S.Q[(c - 6) * S.E + el]; return true; }
  if (c < 15) { if (!has_el) return false; *out = S.w[(c - 12) * S.E + el]; return true; }
  if (c < 18) {
    if (j < 1 || !has_el) return false;
    const int comp = c - 15;
    const int ia = comp == 0 ? 2 : (comp == 1 ? 0 : 1), ib = comp == 0 ? 1 : (comp == 1 ? 2 : 0);
    double rab = 0.0, rba = 0.0;
    for (int k = 0; k < 3; ++k) {
      rab += S.Q[(3 * ia + k) * S.E + el] * S.Q[(3 * ib + k) * S.E + el - 1];
      rba += S.Q[(3 * ib + k) * S.E + el] * S.Q[(3 * ia + k) * S.E + el - 1];
    }
    *out = 0.5 * (rab - rba);
    return true;
  }
  if (c < 21) {
    if (!has_el) return false;
    const int a = c - 18;
    double d = 0.0;
    for (int k = 0; k < 3; ++k) d += S.Q[(3 * a + k) * S.E + el] * (S.x[k * S.N + node + 1] - S.x[k * S.N + node]);
    *out = d;
    return true;
  }
  *out = act[(c - 21) * nwin + b];
  return true;
}

// The 24 input features of node position j of rod b (raw_feature's channels), shifted, scaled
// and rounded to BF16 pairs (channels 24..31 zero), evaluated in FP32 from the FP64 state: the
// network sees 8 bits of each after the shift and scale, against which the FP32 evaluation
// errs by about 2^-20 of the raw value.  The element's edge x_{j+1} - x_j is differenced in
// FP64 first: it carries the stretch strain, ~1e-4 of the edge, which FP32 positions of size
// ~1 would not resolve.  FP64 -> FP32 conversions on the integer pipe (rod_fp.h).  Training
// (features_kernel) and inference (tc_apply_kernel) both use it.
__device__ __forceinline__ void scaled_features(const WinState& S, const double* act3, const Scales& sc, int b, int j,
                                                uint32_t pk[kC0 / 2]) {
  const int64_t node = static_cast<int64_t>(b) * kPos + j, node0 = static_cast<int64_t>(b) * kPos;
  const int64_t el = static_cast<int64_t>(b) * (kPos - 1) + j;
  const bool has_el = j < kPos - 1, has_vor = has_el && j >= 1;
  float f[kFeat];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    f[c] = f32_rn(S.x[c * S.N + node]) - f32_rn(S.x[c * S.N + node0]);
    f[3 + c] = f32_rn(S.v[c * S.N + node]);
    f[21 + c] = f32_rn(act3[c]);
  }
#pragma unroll
  for (int c = 6; c < 21; ++c) f[c] = 0.f;
  if (has_el) {
    float q[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) q[a] = f32_rn(S.Q[a * S.E + el]);
#pragma unroll
    for (int c = 0; c < 6; ++c) f[6 + c] = q[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) f[12 + c] = f32_rn(S.w[c * S.E + el]);
    float l[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) l[k] = f32_rn(S.x[k * S.N + node + 1] - S.x[k * S.N + node]);
#pragma unroll
    for (int a = 0; a < 3; ++a) f[18 + a] = q[3 * a] * l[0] + q[3 * a + 1] * l[1] + q[3 * a + 2] * l[2];
    if (has_vor) {
      // half the axial vector of R - R^T, R_ab = d_a(j) . d_b(j - 1)
      float p[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) p[a] = f32_rn(S.Q[a * S.E + el - 1]);
      auto r = [&](int ia, int ib) { return q[3 * ia] * p[3 * ib] + q[3 * ia + 1] * p[3 * ib + 1] + q[3 * ia + 2] * p[3 * ib + 2]; };
      f[15] = 0.5f * (r(2, 1) - r(1, 2));
      f[16] = 0.5f * (r(0, 2) - r(2, 0));
      f[17] = 0.5f * (r(1, 0) - r(0, 1));
    }
  }
#pragma unroll
  for (int cp = 0; cp < kC0 / 2; ++cp) {
    float h[2] = {0.f, 0.f};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const int c = 2 * cp + t;
      if (c >= kFeat) continue;
      const bool defined = (c < 6 || c >= 21) || (c < 15 || c >= 18 ? has_el : has_vor);
      if (defined) h[t] = (f[c] - sc.in_shift_f[c]) * sc.in_scale[c];
    }
    pk[cp] = pack_bf16(__float2bfloat16_rn(h[0]), __float2bfloat16_rn(h[1]));
  }
}

// features[b][row][c] (BF16), row = position + 2, channels 24..31 and padding rows zero; one
// thread per row
__global__ void features_kernel(WinState S, const double* __restrict__ act, int nwin, Scales sc,
                                __nv_bfloat16* __restrict__ feat) {
  const int b = blockIdx.x, row = threadIdx.x;
  if (b >= nwin || row >= kRows) return;
  const int j = row - 2;
  uint32_t pk[kC0 / 2];
  if (j >= 0 && j < kPos) {
    const double a3[3] = {act[b], act[nwin + b], act[2 * nwin + b]};
    scaled_features(S, a3, sc, b, j, pk);
  } else {
#pragma unroll
    for (int i = 0; i < kC0 / 2; ++i) pk[i] = 0u;
  }
  uint4* dst = reinterpret_cast<uint4*>(feat + (static_cast<int64_t>(b) * kRows + row) * kC0);
#pragma unroll
  for (int i = 0; i < kC0 / 8; ++i) dst[i] = make_uint4(pk[4 * i], pk[4 * i + 1], pk[4 * i + 2], pk[4 * i + 3]);
}

// Training target channel c at node position j of window b (unscaled):
//   0..2 x1 - x0 - T v0     3..5 v1 - v0     6..11 rows d1, d2 of Q1 - exp([-T w0]x) Q0     12..14 w1 - w0
// (element channels are zero at j = 50)
__device__ double target_value(const WinState& A, const WinState& B, double T, double Tq, bool keep_v, bool keep_w, int b,
                               int j, int c) {
  const int64_t node = static_cast<int64_t>(b) * kPos + j, el = static_cast<int64_t>(b) * (kPos - 1) + j;
  const bool has_el = j < kPos - 1;
  if (c < 3) return B.x[c * A.N + node] - A.x[c * A.N + node] - T * A.v[c * A.N + node];  // T = 0: no prior
  if (c < 6) return B.v[(c - 3) * A.N + node] - (keep_v ? A.v[(c - 3) * A.N + node] : 0.0);
  if (!has_el) return 0.0;
  if (c < 12) {
    double q0[9], qp[6];
    const double w0[3] = {A.w[el], A.w[A.E + el], A.w[2 * A.E + el]};
    load_q(A.Q, A.E, el, q0);
    rotate_directors(w0, Tq, q0, qp);
    return B.Q[(c - 6) * A.E + el] - qp[c - 6];
  }
  return B.w[(c - 12) * A.E + el] - (keep_w ? A.w[(c - 12) * A.E + el] : 0.0);
}

// scaled FP32 training targets [b][j][16]
__global__ void targets_kernel(WinState A, WinState B, int nwin, Scales sc, float* __restrict__ tgt) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<int64_t>(nwin) * kPos * kCO) return;
  const int c = i % kCO;
  const int64_t bj = i / kCO;
  const int b = static_cast<int>(bj / kPos), j = static_cast<int>(bj % kPos);
  tgt[i] = (c < kOut) ? static_cast<float>(target_value(A, B, sc.prior_x ? sc.T : 0.0, sc.prior_q ? sc.T : 0.0, sc.keep_v, sc.keep_w, b, j, c) /
                                            sc.out[c])
                      : 0.f;
}

// unscaled FP64 features [b][c][j] (zero where undefined) and mask (1 where defined)
__global__ void raw_features_kernel(WinState S, const double* __restrict__ act, int nwin, double* __restrict__ out,
                                    int8_t* __restrict__ mask) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<int64_t>(nwin) * kFeat * kPos) return;
  const int j = static_cast<int>(i % kPos);
  const int c = static_cast<int>((i / kPos) % kFeat);
  const int b = static_cast<int>(i / (static_cast<int64_t>(kPos) * kFeat));
  double d = 0.0;
  const bool ok = raw_feature(S, act, nwin, b, j, c, &d);
  out[i] = ok ? d : 0.0;
  if (mask) mask[i] = ok ? 1 : 0;
}

// unscaled FP64 targets [b][c][j]: state change minus the kinematic prior
__global__ void raw_targets_kernel(WinState A, WinState B, int nwin, double T, double Tq, int keep_v, int keep_w,
                                   double* __restrict__ out) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<int64_t>(nwin) * kOut * kPos) return;
  const int j = static_cast<int>(i % kPos);
  const int c = static_cast<int>((i / kPos) % kOut);
  const int b = static_cast<int>(i / (static_cast<int64_t>(kPos) * kOut));
  out[i] = target_value(A, B, T, Tq, keep_v, keep_w, b, j, c);
}

// loss = mean (out - tgt)^2 over windows x positions x 15 channels; gradient to BF16 rows
__global__ void loss_kernel(const float* __restrict__ out, const float* __restrict__ tgt, int nwin,
                            __nv_bfloat16* __restrict__ gout, float* __restrict__ loss_sum, float inv_count) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t total = static_cast<int64_t>(nwin) * kRows * kCO;
  float local = 0.f;
  if (i < total) {
    const int c = i % kCO;
    const int64_t brow = i / kCO;
    const int b = static_cast<int>(brow / kRows), row = static_cast<int>(brow % kRows);
    const int j = row - 2;
    float gval = 0.f;
    if (j >= 0 && j < kPos && c < kOut) {
      const int64_t k = (static_cast<int64_t>(b) * kPos + j) * kCO + c;
      const float r = out[k] - tgt[k];
      local = r * r;
      gval = 2.f * r * inv_count;
    }
    gout[i] = __float2bfloat16_rn(gval);
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local != 0.f) atomicAdd(loss_sum, local * inv_count);
}

// New state of node position j of window b: prior + scale * out (FP64); the directors are
// re-orthonormalised (Gram-Schmidt on d1, d2; d3 = d1 x d2); a clamped rod keeps node 0 and
// element 0 as they are, at rest.  Reads the old state from S (window b, may be a shared-memory
// copy), writes the new one to the global arrays at node ng / element eg.
__device__ __forceinline__ void update_node(const WinState& S, int b, int j, const float* __restrict__ o, const Scales& sc,
                                            bool clamped, double* x, double* v, double* Q, double* w, int64_t N,
                                            int64_t E, int64_t ng, int64_t eg) {
  const int64_t node = static_cast<int64_t>(b) * kPos + j;
  const bool held = clamped && j == 0;
  if (!held) {
    for (int c = 0; c < 3; ++c) {
      const double x0 = S.x[c * S.N + node], v0 = S.v[c * S.N + node];
      x[c * N + ng] = fma(sc.out[c], f64_of(o[c]), sc.prior_x ? fma(sc.T, v0, x0) : x0);
      v[c * N + ng] = (sc.keep_v ? v0 : 0.0) + sc.out[3 + c] * f64_of(o[3 + c]);
    }
  } else {
    for (int c = 0; c < 3; ++c) {
      x[c * N + ng] = S.x[c * S.N + node];
      v[c * N + ng] = 0.0;
    }
  }
  if (j >= kPos - 1) return;
  const int64_t e = static_cast<int64_t>(b) * (kPos - 1) + j;
  double q0[9];
  load_q(S.Q, S.E, e, q0);
  if (held) {
    for (int a = 0; a < 9; ++a) Q[a * E + eg] = q0[a];
    for (int c = 0; c < 3; ++c) w[c * E + eg] = 0.0;
    return;
  }
  double qp[6];
  const double w0[3] = {S.w[e], S.w[S.E + e], S.w[2 * S.E + e]};
  rotate_directors(w0, sc.prior_q ? sc.T : 0.0, q0, qp);
  double d1[3], d2[3];
  for (int c = 0; c < 3; ++c) {
    d1[c] = qp[c] + sc.out[6 + c] * f64_of(o[6 + c]);
    d2[c] = qp[3 + c] + sc.out[9 + c] * f64_of(o[9 + c]);
    w[c * E + eg] = (sc.keep_w ? w0[c] : 0.0) + sc.out[12 + c] * f64_of(o[12 + c]);
  }
  const double n1 = rsqrt_nr(fma(d1[0], d1[0], fma(d1[1], d1[1], d1[2] * d1[2])));
  for (int c = 0; c < 3; ++c) d1[c] *= n1;
  const double p = fma(d1[0], d2[0], fma(d1[1], d2[1], d1[2] * d2[2]));
  for (int c = 0; c < 3; ++c) d2[c] = fma(-p, d1[c], d2[c]);
  const double n2 = rsqrt_nr(fma(d2[0], d2[0], fma(d2[1], d2[1], d2[2] * d2[2])));
  for (int c = 0; c < 3; ++c) d2[c] *= n2;
  const double d3[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2], d1[0] * d2[1] - d1[1] * d2[0]};
  for (int c = 0; c < 3; ++c) {
    Q[c * E + eg] = d1[c];
    Q[(3 + c) * E + eg] = d2[c];
    Q[(6 + c) * E + eg] = d3[c];
  }
}

// Noise-injected training-window start (the surrogate's training; the paper has no
// counterpart): out = in plus noise x spread x r for positions (r: rx), velocities (rv) and
// angular velocities (rw); directors turned to first order by the lab-frame angle vector
// noise x turn x ra, d_a + ang x d_a for d1 and d2, then Gram-Schmidt and d3 = d1 x d2; the node
// 0 and element 0 of a held window keep their position and directors with zero rates.  The
// normal draws r are inputs.  noise = 0 re-orthonormalises the directors alone.
struct Spread {
  double s[kOut];
  double turn;   // largest director scale
};

__global__ void perturb_kernel(WinState S, int nwin, const double* __restrict__ rx, const double* __restrict__ rv,
                               const double* __restrict__ rw, const double* __restrict__ ra, Spread sp, double noise,
                               const int8_t* __restrict__ held, double* __restrict__ x, double* __restrict__ v,
                               double* __restrict__ Q, double* __restrict__ w) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<int64_t>(nwin) * kPos) return;
  const int b = static_cast<int>(i / kPos), j = static_cast<int>(i % kPos);
  const bool hold = held && held[b] && j == 0;
  for (int c = 0; c < 3; ++c) {
    const int64_t k = c * S.N + i;
    x[k] = hold ? S.x[k] : fma(noise * sp.s[c], rx[k], S.x[k]);
    v[k] = hold ? 0.0 : fma(noise * sp.s[3 + c], rv[k], S.v[k]);
  }
  if (j >= kPos - 1) return;
  const int64_t e = static_cast<int64_t>(b) * (kPos - 1) + j;
  if (hold) {
    for (int a = 0; a < 9; ++a) Q[a * S.E + e] = S.Q[a * S.E + e];
    for (int c = 0; c < 3; ++c) w[c * S.E + e] = 0.0;
    return;
  }
  double ang[3], d1[3], d2[3];
  for (int c = 0; c < 3; ++c) {
    w[c * S.E + e] = fma(noise * sp.s[12 + c], rw[c * S.E + e], S.w[c * S.E + e]);
    ang[c] = noise * sp.turn * ra[c * S.E + e];
    d1[c] = S.Q[c * S.E + e];
    d2[c] = S.Q[(3 + c) * S.E + e];
  }
  const double t1[3] = {ang[1] * d1[2] - ang[2] * d1[1], ang[2] * d1[0] - ang[0] * d1[2], ang[0] * d1[1] - ang[1] * d1[0]};
  const double t2[3] = {ang[1] * d2[2] - ang[2] * d2[1], ang[2] * d2[0] - ang[0] * d2[2], ang[0] * d2[1] - ang[1] * d2[0]};
  for (int c = 0; c < 3; ++c) {
    d1[c] += t1[c];
    d2[c] += t2[c];
  }
  const double n1 = 1.0 / sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
  for (int c = 0; c < 3; ++c) d1[c] *= n1;
  const double p = d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2];
  for (int c = 0; c < 3; ++c) d2[c] -= p * d1[c];
  const double n2 = 1.0 / sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
  for (int c = 0; c < 3; ++c) d2[c] *= n2;
  const double d3[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2], d1[0] * d2[1] - d1[1] * d2[0]};
  for (int c = 0; c < 3; ++c) {
    Q[c * S.E + e] = d1[c];
    Q[(3 + c) * S.E + e] = d2[c];
    Q[(6 + c) * S.E + e] = d3[c];
  }
}

// unfused update of every node position from the network output [nrods][51][16] (in place)
__global__ void apply_kernel(double* x, double* v, double* Q, double* w, int64_t N, int64_t E, int nrods,
                             const float* __restrict__ out, Scales sc, const RodConst* __restrict__ rods) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<int64_t>(nrods) * kPos) return;
  const int b = static_cast<int>(i / kPos), j = static_cast<int>(i % kPos);
  WinState S;
  S.x = x;
  S.v = v;
  S.Q = Q;
  S.w = w;
  S.N = N;
  S.E = E;
  update_node(S, b, j, out + i * kCO, sc, rods[b].clamp != 0, x, v, Q, w, N, E, i,
              static_cast<int64_t>(b) * (kPos - 1) + j);
}

// Copy the state of the sampled rods sample[0..n) of a system into a system that holds just
// those rods (same order, 50 elements each).
__global__ void gather_rods_kernel(const double* __restrict__ x, const double* __restrict__ v, const double* __restrict__ Q,
                                   const double* __restrict__ w, int64_t N, int64_t E, const int32_t* __restrict__ sample,
                                   int n, double* __restrict__ xs, double* __restrict__ vs, double* __restrict__ Qs,
                                   double* __restrict__ ws) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<int64_t>(n) * kPos) return;
  const int k = static_cast<int>(i / kPos), j = static_cast<int>(i % kPos);
  const int64_t Ns = static_cast<int64_t>(n) * kPos, Es = static_cast<int64_t>(n) * (kPos - 1);
  const int64_t src = static_cast<int64_t>(sample[k]) * kPos + j;
  for (int c = 0; c < 3; ++c) {
    xs[c * Ns + i] = x[c * N + src];
    vs[c * Ns + i] = v[c * N + src];
  }
  if (j < kPos - 1) {
    const int64_t se = static_cast<int64_t>(sample[k]) * (kPos - 1) + j, de = static_cast<int64_t>(k) * (kPos - 1) + j;
    for (int a = 0; a < 9; ++a) Qs[a * Es + de] = Q[a * E + se];
    for (int c = 0; c < 3; ++c) ws[c * Es + de] = w[c * E + se];
  }
}

// tips[k][c] = tip position of sampled rod k
__global__ void save_tips_kernel(const double* __restrict__ x, int64_t N, const int32_t* __restrict__ sample, int n,
                                 double* __restrict__ tips) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t tip = static_cast<int64_t>(sample[k]) * kPos + kPos - 1;
  for (int c = 0; c < 3; ++c) tips[3 * k + c] = x[c * N + tip];
}

// max over k of |tip of rod k of a shadow system - tips[k]| / L_k (as non-negative double bits)
__global__ void local_error_kernel(const double* __restrict__ xs, int64_t Ns, const double* __restrict__ tips, int n,
                                   const double* __restrict__ rest_len_s, unsigned long long* err_bits) {
  double worst = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int64_t tip = static_cast<int64_t>(k) * kPos + kPos - 1;
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double d = xs[c * Ns + tip] - tips[3 * k + c];
      d2 += d * d;
    }
    double L = 0.0;
    for (int q = 0; q < kPos - 1; ++q) L += rest_len_s[static_cast<int64_t>(k) * (kPos - 1) + q];
    double e = sqrt(d2) / L;
    if (!(e <= 1e300)) e = INFINITY;
    worst = fmax(worst, e);
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) atomicMax(err_bits, static_cast<unsigned long long>(__double_as_longlong(worst)));
}

// ---- fused inference on the fifth-generation tensor cores (tcgen05)
//
// One persistent block per SM keeps the four layers' BF16 weights in shared memory and runs two
// independent pipelines of 256 threads, each walking its own groups of four windows (rods).  A
// group's activations live in the pipeline's shared-memory store of rows, two 128-row tiles of
// two windows each: window slot i of a tile takes rows 53 i .. 53 i + 52 of it, two zero rows
// and then its 51 node positions, so the two zero rows in front of a window are the right-hand
// padding of the window before it as well (rows 106..127 of a tile stay zero).  A convolution
// layer is then one GEMM per tile,
//   D[m][o] = sum_t sum_c S[m + t][c] W[o][t c],   t = 0..4,
// where output row m (slot m / 53, position m % 53, an output where that is below 51) reads
// store rows m .. m + 4, i.e. the positions m % 53 - 2 .. m % 53 + 2 of its own window.  The
// store is K-major with consecutive rows 16 bytes apart inside each block of 8 channels (core
// matrices of 8 consecutive rows, row-group stride 128 bytes, channel-block stride one whole
// column block of the store), so the A operand of tap t is the store seen from row t -- its
// descriptor starts 16 t bytes further on -- and no im2col copy is made.  A tile's outputs read
// only its own rows, so each tile -- its four warps, warp w reading lanes 32 (w % 4) .. + 31 of
// the tile's 64 accumulator columns in tensor memory -- runs the layers on its own: its first
// thread issues the tile's MMAs (tap x 16 input channels) and commits them to the tile's
// mbarrier, the warps wait, add the bias, apply SiLU, round to BF16 and write their rows back
// into the store as the next layer's input (store row m + 2), and meet at the tile's own named
// barrier before the next layer; one tile's epilogue runs while the other's MMAs do.  The output layer's epilogue leaves the 16 outputs of each node position in
// shared memory.  The FP64 work -- the features (computed one thread per node position from the
// state in global memory) and the update of the state in place (one thread per node position;
// update_node reads only that node and the element starting there) -- runs in separate phases,
// which the ping-pong schedule below sets against the other pipeline's tensor-core phases: on
// this part the SM executes 2 FP64 lanes per cycle against 128 FP32 lanes, and the two kinds of
// work use different units.  Waits are bounded: a wait
// that runs out latches ERR_TIMEOUT into the system's error word, waits once more for the MMAs
// in flight, and the pipeline passes the rest of its phases idle; the block frees the tensor
// memory and ends.
constexpr int kPipes = 2;                        // independent pipelines per block
constexpr int kTiles = 2;                        // 128-row tiles per group
constexpr int kTM = 128;
constexpr int kWS = kPos + 2;                    // store rows per window (53)
constexpr int kWPT = kTM / kWS;                  // windows per tile (2): no window crosses a tile
constexpr int kGW = kTiles * kWPT;               // windows per group (4)
constexpr int kSR = kTiles * kTM + kTaps - 1;    // store rows (260): the last tile reads 4 rows past it
constexpr uint32_t kChunk = kSR * 16;            // bytes of one block of 8 channels of a store
constexpr uint32_t kCoreK = 128;                 // K-direction stride of the weights' core matrices
constexpr uint32_t kRowW = kTaps * kC * 16;      // row-group stride of W2..W4 (K = 320)
constexpr uint32_t kRowW1 = kTaps * kC0 * 16;    // row-group stride of W1 (K = 160)
constexpr size_t kTcS = size_t(kC / 8) * kChunk;
constexpr size_t kTcW1 = size_t(kC) * kTaps * kC0 * 2;
constexpr size_t kTcW2 = size_t(kC) * kTaps * kC * 2;
constexpr size_t kTcW4 = size_t(kCO) * kTaps * kC * 2;
constexpr size_t kTcBias = size_t(3 * kC + kCO) * 4;
constexpr size_t kTcOut = size_t(kGW) * kPos * kCO * 4;   // a pipeline's outputs of one group
constexpr size_t kTcActS = size_t(kPipes) * 2 * kGW * 3 * 8;
constexpr size_t kTcSmem = kPipes * (kTcS + kTcOut) + kTcW1 + 2 * kTcW2 + kTcW4 + kTcBias + kTcActS;
constexpr int kPipeThreads = 32 * 4 * kTiles;    // a pipeline's warp w: lane quadrant w % 4 of tile w / 4
constexpr int kTcThreads = kPipes * kPipeThreads;
constexpr uint32_t kTmemCols = 64 * kTiles * kPipes;
constexpr uint32_t kWaitPolls = 1u << 20;        // polls of an mbarrier wait before it gives up
static_assert(kTcSmem <= 227 * 1024, "the fused kernel's shared memory exceeds a block's");
static_assert(kTcS % 16 == 0 && kTcW1 % 16 == 0 && kTcW2 % 16 == 0 && kTcW4 % 16 == 0, "16-byte operands");
static_assert(kTcOut % 16 == 0, "16-byte output rows");
static_assert((kPipes * (kTcS + kTcOut) + kTcW1 + 2 * kTcW2 + kTcW4 + kTcBias) % 8 == 0, "aligned base-couple samples");
static_assert((kWPT - 1) * kWS + (kPos - 1) + (kTaps - 1) + 2 < kTM,
              "a tile's outputs read only its own rows: the tiles' layers are independent");
static_assert(kGW * kPos + kGW * 3 <= kPipeThreads, "one thread per node position, the rest for the base couple");
static_assert((kTmemCols & (kTmemCols - 1)) == 0 && kTmemCols >= 32, "tensor-memory allocation size");

// byte offset of channel c of store row r
__device__ __forceinline__ uint32_t store_off(int r, int c) {
  return static_cast<uint32_t>(c >> 3) * kChunk + static_cast<uint32_t>(r) * 16u + static_cast<uint32_t>(c & 7) * 2u;
}

// Debug capture of one call (rod_surrogate_apply_debug): per layer l, window b, position p and
// channel o, pre[((l R + b) 51 + p) 64 + o] = accumulator + bias, act[same] = the BF16 input of
// layer l (l = 0: the features), widened.
struct TcDebug {
  float* pre;
  float* act;
};

__device__ __forceinline__ void tc_debug_put(float* a, int l, int nrods, int b, int p, int o, float val) {
  a[((static_cast<int64_t>(l) * nrods + b) * kPos + p) * kC + o] = val;
}

__global__ void __launch_bounds__(kTcThreads, 1) tc_apply_kernel(double* x, double* v, double* Q, double* w,
                                                                  int64_t N, int64_t E, int nrods,
                                                                  const RodConst* __restrict__ rods, double t,
                                                                  Scales sc, const __nv_bfloat16* __restrict__ wf,
                                                                  const float* __restrict__ master, int* err,
                                                                  uint32_t wait_polls, TcDebug dbg) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sW1 = smem_raw + kPipes * (kTcS + kTcOut);
  unsigned char* sW2 = sW1 + kTcW1;
  unsigned char* sW3 = sW2 + kTcW2;
  unsigned char* sW4 = sW3 + kTcW2;
  float* bias = reinterpret_cast<float*>(sW4 + kTcW4);
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[kPipes * kTiles];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // the stores zero (rows that are no node position stay so), the weights in the K-major
  // core-matrix layout, the biases
  for (int i = tid; i < static_cast<int>(kPipes * kTcS / 16); i += blockDim.x)
    reinterpret_cast<uint4*>(smem_raw)[i] = make_uint4(0u, 0u, 0u, 0u);
  {
    const __nv_bfloat16* src[4] = {wf, wf + kW1, wf + kW1 + kW2, wf + kW1 + kW2 + kW3};
    unsigned char* dst[4] = {sW1, sW2, sW3, sW4};
    const int rows[4] = {kC, kC, kC, kCO}, kk[4] = {kTaps * kC0, kTaps * kC, kTaps * kC, kTaps * kC};
    const uint32_t rs[4] = {kRowW1, kRowW, kRowW, kRowW};
    for (int l = 0; l < 4; ++l)
      for (int i = tid; i < rows[l] * kk[l] / 8; i += blockDim.x) {  // chunks of 8 elements of K
        const int r = (8 * i) / kk[l], k = (8 * i) % kk[l];
        *reinterpret_cast<uint4*>(dst[l] + tc::kmajor_offset(r, k, kCoreK, rs[l])) =
            *reinterpret_cast<const uint4*>(src[l] + static_cast<int64_t>(r) * kk[l] + k);
      }
    for (int i = tid; i < kC; i += blockDim.x) {
      bias[i] = master[kOffB1 + i];
      bias[kC + i] = master[kOffB2 + i];
      bias[2 * kC + i] = master[kOffB3 + i];
    }
    for (int i = tid; i < kCO; i += blockDim.x) bias[3 * kC + i] = master[kOffB4 + i];
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0)
    for (int p = 0; p < kPipes * kTiles; ++p) tc::mbar_init(&mbar[p], 1);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();

  // From here on each pipeline (kPipeThreads consecutive threads) walks its own groups with its
  // own store, accumulator columns, mbarrier and named barrier; the two meet again only at the
  // end, so one pipeline's FP64 work overlaps the other's MMAs and epilogues.
  const int pipe = tid / kPipeThreads, ptid = tid % kPipeThreads;
  const uint32_t bar_id = 1u + static_cast<uint32_t>(pipe);
  unsigned char* sS = smem_raw + pipe * kTcS;
  float4* outs = reinterpret_cast<float4*>(smem_raw + kPipes * kTcS + pipe * kTcOut);  // [c / 4][node]
  double* act_s = reinterpret_cast<double*>(bias + 3 * kC + kCO) + pipe * 2 * kGW * 3;  // [group & 1][window][3]

  const uint32_t tcol = static_cast<uint32_t>(64 * kTiles * pipe);   // the pipeline's first accumulator column
  uint32_t phase = 0;
  const int wl = ptid >> 5;
  const int q = wl & 3, g = wl >> 2;             // lane quadrant (= warp % 4) and tile of this warp's rows
  const int m = kTM * g + 32 * q + lane;         // the output row of this thread
  const int slot = (32 * q + lane) / kWS;        // its window slot in the tile
  const int mw = kWPT * g + slot, mp = (32 * q + lane) % kWS;   // its window in the group, node position
  const bool row_pos = slot < kWPT && mp < kPos; // a node position (of a window slot of the group)
  // each tile (its four warps) runs the layers on its own: own barrier, mbarrier, issuing thread
  const uint32_t tbar = 4u + static_cast<uint32_t>(kTiles * pipe + g);
  uint64_t* mb = &mbar[kTiles * pipe + g];
  const bool issuer = (32 * q + lane) == 0;
  const uint32_t tmem = tmem_base;
  const uint32_t tacc = tmem + (static_cast<uint32_t>(32 * q) << 16) + tcol + 64u * static_cast<uint32_t>(g);
  WinState S;                                    // the system's state, read in place
  S.x = x;
  S.v = v;
  S.Q = Q;
  S.w = w;
  S.N = N;
  S.E = E;

  // Issue layer l's MMAs (the pipeline's first thread) after every thread's writes to the store
  // are visible to the tensor cores and every read of the accumulators is done; wait for them.
  // False when a wait ran out (the error is latched and the MMAs in flight drained).
  // wait_polls with the top bit set (a test of the timeout path): issue nothing, so that the
  // wait runs out after the remaining bits' polls.
  const bool no_issue = (wait_polls & 0x80000000u) != 0u;
  const uint32_t polls = wait_polls & 0x7FFFFFFFu;
  auto run_layer = [&](int l) -> bool {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    tc::bar_sync(tbar, 128);
    if (issuer && !no_issue) {
      tc::fence_after_sync();
      const uint32_t s0 = tc::smem_addr(sS);
      const int cin = l == 0 ? kC0 : kC;
      const uint32_t id = tc::idesc_bf16_f32(kTM, l == 3 ? kCO : kC);
      const uint32_t w0 = tc::smem_addr(l == 0 ? sW1 : (l == 1 ? sW2 : (l == 2 ? sW3 : sW4)));
      const uint32_t rw = l == 0 ? kRowW1 : kRowW;
      int s = 0;
      for (int tp = 0; tp < kTaps; ++tp)
        for (int h = 0; h < cin / 16; ++h, ++s)
          tc::mma_bf16(tmem + tcol + 64u * g,
                       tc::smem_desc(s0 + static_cast<uint32_t>(kTM * g + tp) * 16u + 2u * h * kChunk, kChunk, 128u),
                       tc::smem_desc(w0 + static_cast<uint32_t>((tp * cin + 16 * h) / 8) * kCoreK, kCoreK, rw), id,
                       s > 0);
      tc::commit(mb);
    }
    const bool ok = tc::mbar_wait(mb, phase, polls);
    if (tc::bar_or(tbar, 128, !ok)) {
      if (issuer) atomicOr(err, ERR_TIMEOUT);
      tc::mbar_wait(mb, phase, no_issue ? polls : kWaitPolls);  // the MMAs in flight finish first
      return false;
    }
    phase ^= 1u;
    tc::fence_after_sync();
    return true;
  };

  // Ping-pong schedule.  Pipeline p's work is a sequence of phases: F0, T0, U0 F1, T1, U1 F2, ...,
  // U(n-1), where Fk computes group k's features (FP64, one thread per node position) into the
  // store, Tk runs its four layers (tensor cores and FP32 epilogues; the outputs go to shared
  // memory) and Uk updates its node positions (FP64, one thread per node position).  Pipeline 1
  // runs one phase behind pipeline 0 and the whole block meets at a barrier after every phase,
  // so each FP64 phase of one pipeline coincides with a tensor-core phase of the other.  Every
  // thread passes the same number of these barriers (a pipeline with fewer groups, or one whose
  // wait ran out, passes them idle).
  const int ngroups = (nrods + kGW - 1) / kGW;
  const int gstride = gridDim.x * kPipes;
  auto groups_of = [&](int p) {
    const int g0 = blockIdx.x * kPipes + p;
    return g0 < ngroups ? (ngroups - 1 - g0) / gstride + 1 : 0;
  };
  auto first_rod = [&](int k) { return (blockIdx.x * kPipes + pipe + k * gstride) * kGW; };
  // base couple of each window of group k at its start, middle and end, by the threads past
  // the node positions
  auto couple_samples = [&](int k) {
    const int i = ptid - kGW * kPos, b0 = first_rod(k);
    if (i >= 0 && i < min(kGW, nrods - b0) * 3) {
      const RodConst& rc = rods[b0 + i / 3];
      act_s[(k & 1) * kGW * 3 + i] = rc.act_amp * sin(rc.act_omega * (t + 0.5 * (i % 3) * sc.T) + rc.act_phase);
    }
  };
  const int nmine = groups_of(pipe), nmax = groups_of(0);   // pipeline 0 has the most
  if (nmine > 0) couple_samples(0);
  tc::bar_sync(bar_id, kPipeThreads);
  bool alive = true;
  for (int slot = 0; slot <= 2 * nmax + 1; ++slot) {
    const int ph = slot - pipe;                  // this pipeline's phase index
    if (alive && ph >= 0 && ph <= 2 * nmine) {
      const int k = ph >> 1;                     // the group of a T phase, the group of F in an U F phase
      const int b0 = first_rod(k);
      const int nw = min(kGW, nrods - b0);
      if (ph & 1) {
        // Tk: three hidden layers (accumulator + bias -> SiLU -> BF16 into the store), output layer
        for (int l = 0; l < 3 && alive; ++l) {
          if (!(alive = run_layer(l))) break;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            uint32_t r[2][16];
            tc::ld16(tacc + 32u * half, r[0]);
            tc::ld16(tacc + 32u * half + 16u, r[1]);
            tc::ld_wait();
            if (row_pos) {
              uint32_t pk[16];
#pragma unroll
              for (int c = 0; c < 32; c += 2) {
                const int oc = 32 * half + c;
                const float p0 = __uint_as_float(r[c >> 4][c & 15]) + bias[l * kC + oc];
                const float p1 = __uint_as_float(r[c >> 4][(c & 15) + 1]) + bias[l * kC + oc + 1];
                const __nv_bfloat16 a0 = __float2bfloat16_rn(silu(p0)), a1 = __float2bfloat16_rn(silu(p1));
                pk[c / 2] = pack_bf16(a0, a1);
                if (dbg.pre && mw < nw) {
                  tc_debug_put(dbg.pre, l, nrods, b0 + mw, mp, oc, p0);
                  tc_debug_put(dbg.pre, l, nrods, b0 + mw, mp, oc + 1, p1);
                  tc_debug_put(dbg.act, l + 1, nrods, b0 + mw, mp, oc, __bfloat162float(a0));
                  tc_debug_put(dbg.act, l + 1, nrods, b0 + mw, mp, oc + 1, __bfloat162float(a1));
                }
              }
#pragma unroll
              for (int cb = 0; cb < 4; ++cb)
                *reinterpret_cast<uint4*>(sS + store_off(m + 2, 32 * half + 8 * cb)) =
                    make_uint4(pk[4 * cb], pk[4 * cb + 1], pk[4 * cb + 2], pk[4 * cb + 3]);
            }
          }
        }
        if (alive) alive = run_layer(3);
        if (alive) {
          uint32_t r[16];
          tc::ld16(tacc, r);
          tc::ld_wait();
          if (row_pos && mw < nw) {
            float o[kCO];
#pragma unroll
            for (int c = 0; c < kCO; ++c) o[c] = __uint_as_float(r[c]) + bias[3 * kC + c];
            const int node = mw * kPos + mp;
#pragma unroll
            for (int c4 = 0; c4 < kCO / 4; ++c4)
              outs[c4 * kGW * kPos + node] = make_float4(o[4 * c4], o[4 * c4 + 1], o[4 * c4 + 2], o[4 * c4 + 3]);
            if (dbg.pre)
              for (int c = 0; c < kCO; ++c) tc_debug_put(dbg.pre, 3, nrods, b0 + mw, mp, c, o[c]);
          }
        }
        // a wait that ran out in either tile stops the whole pipeline
        alive = !tc::bar_or(bar_id, kPipeThreads, !alive);
      } else {
        // Fk first (its stores go to shared memory, so the update's global loads below may be
        // issued under its arithmetic), then U(k-1)
        if (k < nmine) {
          // Fk: the features, one thread per node position (a window slot past the last rod gets
          // zeros); the threads past them take the next group's base-couple samples
          if (ptid < kGW * kPos) {
            const int wi = ptid / kPos, j = ptid % kPos;
            uint32_t pk[kC0 / 2];
            if (wi < nw) {
              scaled_features(S, act_s + (k & 1) * kGW * 3 + 3 * wi, sc, b0 + wi, j, pk);
            } else {
#pragma unroll
              for (int i = 0; i < kC0 / 2; ++i) pk[i] = 0u;
            }
            const int r = kTM * (wi / kWPT) + kWS * (wi % kWPT) + j + 2;
#pragma unroll
            for (int cb = 0; cb < kC0 / 8; ++cb)
              *reinterpret_cast<uint4*>(sS + store_off(r, 8 * cb)) =
                  make_uint4(pk[4 * cb], pk[4 * cb + 1], pk[4 * cb + 2], pk[4 * cb + 3]);
            if (dbg.act && wi < nw)
              for (int c = 0; c < kC0; ++c)
                tc_debug_put(dbg.act, 0, nrods, b0 + wi, j, c,
                             __bfloat162float(__ushort_as_bfloat16(static_cast<unsigned short>(pk[c / 2] >> (16 * (c & 1))))));
          } else if (k + 1 < nmine) {
            couple_samples(k + 1);
          }
        }
        // U(k-1): the FP64 update of the previous group's node positions
        if (k > 0) {
          const int bp = first_rod(k - 1);
          if (ptid < min(kGW, nrods - bp) * kPos) {
            float o[kCO];
#pragma unroll
            for (int c4 = 0; c4 < kCO / 4; ++c4) {
              const float4 f4 = outs[c4 * kGW * kPos + ptid];
              o[4 * c4] = f4.x;
              o[4 * c4 + 1] = f4.y;
              o[4 * c4 + 2] = f4.z;
              o[4 * c4 + 3] = f4.w;
            }
            const int ub = bp + ptid / kPos, j = ptid % kPos;
            update_node(S, ub, j, o, sc, rods[ub].clamp != 0, x, v, Q, w, N, E, static_cast<int64_t>(ub) * kPos + j,
                        static_cast<int64_t>(ub) * (kPos - 1) + j);
          }
        }
      }
    }
    tc::fence_proxy_async();                    // this thread's store writes, for either tile's MMAs
    tc::bar_sync(kPipes + 1, kTcThreads);       // the phase boundary of the whole block
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_free(tmem, kTmemCols);
}

// base couple A sin(omega t + phi) of every rod at t, t + T/2 and t + T
__global__ void actuation_kernel(const RodConst* __restrict__ rods, int nrods, double t, double T, double* __restrict__ act) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrods) return;
  for (int k = 0; k < 3; ++k) {
    const double tk = t + 0.5 * k * T;
    act[k * nrods + r] = rods[r].act_amp * sin(rods[r].act_omega * tk + rods[r].act_phase);
  }
}

// max over sampled rods of |x_tip - x_tip(reference)| / L (L = sum of rest lengths); a
// non-finite distance counts as infinite.  err_bits: the maximum as the bit pattern of a
// non-negative double (monotone as an integer), cleared by the caller.
__global__ void tip_error_kernel(const double* __restrict__ x, int64_t N, const double* __restrict__ xref, int64_t Nref,
                                 const int32_t* __restrict__ sample, int n_sample, const double* __restrict__ rest_len,
                                 unsigned long long* err_bits) {
  double worst = 0.0;
  for (int i = threadIdx.x; i < n_sample; i += blockDim.x) {
    const int64_t r = sample[i];
    const int64_t tip = r * kPos + kPos - 1, tip_ref = static_cast<int64_t>(i) * kPos + kPos - 1;
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double d = x[c * N + tip] - xref[c * Nref + tip_ref];
      d2 += d * d;
    }
    double L = 0.0;
    for (int k = 0; k < kPos - 1; ++k) L += rest_len[r * (kPos - 1) + k];
    double e = sqrt(d2) / L;
    if (!(e <= 1e300)) e = INFINITY;
    worst = fmax(worst, e);
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) atomicMax(err_bits, static_cast<unsigned long long>(__double_as_longlong(worst)));
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m, float* __restrict__ v,
                            int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = gr[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 copies of the FP32 master weights: forward layout [COUT][t*CIN + c] and the tap-transposed
// layout used by the input gradient, Wt[c][t*COUT + o] = W[o][t*CIN + c]
__global__ void cast_weights_kernel(const float* __restrict__ master, __nv_bfloat16* __restrict__ wf,
                                    __nv_bfloat16* __restrict__ wt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int offs[4] = {kOffW1, kOffW2, kOffW3, kOffW4};
  const int cin[4] = {kC0, kC, kC, kC};
  const int cout[4] = {kC, kC, kC, kCO};
  int base = 0;
  for (int l = 0; l < 4; ++l) {
    const int n = cout[l] * kTaps * cin[l];
    if (i >= base && i < base + n) {
      const int k = i - base;
      const int o = k / (kTaps * cin[l]), rem = k % (kTaps * cin[l]);
      const int t = rem / cin[l], c = rem % cin[l];
      const __nv_bfloat16 vb = __float2bfloat16_rn(master[offs[l] + k]);
      wf[base + k] = vb;
      wt[base + (c * kTaps * cout[l] + t * cout[l] + o)] = vb;
    }
    base += n;
  }
}

}  // namespace sur
}  // namespace rod

// ------------------------------------------------------------------------------ host side

using namespace rod;
using namespace rod::sur;

struct rod_surrogate {
  int window = 50;
  double dt = 0.0;
  Scales sc{};
  float *master = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  __nv_bfloat16 *wf = nullptr, *wt = nullptr;   // BF16 forward / transposed weights
  int64_t adam_t = 0;
  // per-batch buffers (grown on demand)
  int cap = 0;
  int last_nwin = 0;  // windows of the last training step (rod_surrogate_debug_buffer)
  uint32_t wait_polls = 0;  // polls of the fused kernel's mbarrier waits (0: the default)
  __nv_bfloat16 *a0 = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr;  // input, hidden 1..3
  float *p1 = nullptr, *p2 = nullptr, *p3 = nullptr;                        // pre-activations
  float *outf = nullptr, *tgt = nullptr, *loss = nullptr;
  float* part = nullptr;   // per-chunk partial weight gradients [chunks][largest layer]
  __nv_bfloat16 *g4 = nullptr, *g3 = nullptr, *g2 = nullptr, *g1 = nullptr;
  double* act = nullptr;
  bool weights_dirty = true;
  // rollout: checkpoint of the system state, sampled rods, error word
  double* ck = nullptr;
  int64_t ck_cap = 0;
  int32_t* sample = nullptr;
  int sample_cap = 0;
  unsigned long long* err_dev = nullptr;
  unsigned long long* err_host = nullptr;  // pinned
  // local checked rollouts: per shadow slot the sampled tips, an error word (device and pinned
  // host) and three events, kept between calls (no allocation inside a rollout)
  struct CheckRes {
    double* tips = nullptr;
    int tips_cap = 0;
    unsigned long long* err_dev = nullptr;
    unsigned long long* err_host = nullptr;
    cudaEvent_t gathered = nullptr, tipped = nullptr, done = nullptr;
  };
  std::vector<CheckRes> chk;
};

namespace {

int64_t bf_off(int layer) {  // offset of layer l's weights in the BF16 weight arrays
  const int64_t n[4] = {kW1, kW2, kW3, kW4};
  int64_t o = 0;
  for (int l = 0; l < layer; ++l) o += n[l];
  return o;
}
constexpr int64_t kBfTotal = kW1 + kW2 + kW3 + kW4;
constexpr int kWgradWindows = 16;   // windows per chunk of the weight gradient

cudaError_t grow(rod_surrogate* s, int nwin) {
  if (nwin <= s->cap) return cudaSuccess;
  void* ptrs[] = {s->a0, s->a1, s->a2, s->a3, s->p1, s->p2, s->p3, s->outf, s->tgt, s->g4, s->g3, s->g2, s->g1, s->act,
                  s->part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  s->cap = 0;
  const size_t rows = static_cast<size_t>(nwin) * kRows;
  cudaError_t e;
  if ((e = cudaMalloc(&s->a0, rows * kC0 * 2)) || (e = cudaMalloc(&s->a1, rows * kC * 2)) ||
      (e = cudaMalloc(&s->a2, rows * kC * 2)) || (e = cudaMalloc(&s->a3, rows * kC * 2)) ||
      (e = cudaMalloc(&s->p1, rows * kC * 4)) || (e = cudaMalloc(&s->p2, rows * kC * 4)) ||
      (e = cudaMalloc(&s->p3, rows * kC * 4)) || (e = cudaMalloc(&s->outf, static_cast<size_t>(nwin) * kPos * kCO * 4)) ||
      (e = cudaMalloc(&s->tgt, static_cast<size_t>(nwin) * kPos * kCO * 4)) || (e = cudaMalloc(&s->g4, rows * kCO * 2)) ||
      (e = cudaMalloc(&s->g3, rows * kC * 2)) || (e = cudaMalloc(&s->g2, rows * kC * 2)) ||
      (e = cudaMalloc(&s->g1, rows * kC * 2)) || (e = cudaMalloc(&s->act, static_cast<size_t>(nwin) * 3 * 8)) ||
      (e = cudaMalloc(&s->part, static_cast<size_t>((nwin + kWgradWindows - 1) / kWgradWindows) * (kW2 + kC) * 4)))
    return e;
  // the kernels write rows 2..57 only: the padding rows must start (and stay) zero
  if ((e = cudaMemset(s->a1, 0, rows * kC * 2)) || (e = cudaMemset(s->a2, 0, rows * kC * 2)) ||
      (e = cudaMemset(s->a3, 0, rows * kC * 2)) || (e = cudaMemset(s->g3, 0, rows * kC * 2)) ||
      (e = cudaMemset(s->g2, 0, rows * kC * 2)) || (e = cudaMemset(s->g1, 0, rows * kC * 2)) ||
      (e = cudaMemset(s->p1, 0, rows * kC * 4)) || (e = cudaMemset(s->p2, 0, rows * kC * 4)) ||
      (e = cudaMemset(s->p3, 0, rows * kC * 4)))
    return e;
  s->cap = nwin;
  return cudaSuccess;
}

cudaError_t refresh_weights(rod_surrogate* s, cudaStream_t st) {
  if (!s->weights_dirty) return cudaSuccess;
  cast_weights_kernel<<<(kBfTotal + 255) / 256, 256, 0, st>>>(s->master, s->wf, s->wt);
  s->weights_dirty = false;
  return cudaGetLastError();
}

// forward through the four layers; features must be in a0; keeps pre-activations when train
cudaError_t forward(rod_surrogate* s, int nwin, bool train, cudaStream_t st) {
  const float* m = s->master;
  conv_kernel<kC0, kC, EPI_HIDDEN, false><<<nwin, 128, 0, st>>>(s->a0, s->wf + bf_off(0), m + kOffB1, s->a1, nullptr,
                                                                 train ? s->p1 : nullptr, nullptr, nwin);
  conv_kernel<kC, kC, EPI_HIDDEN, false><<<nwin, 128, 0, st>>>(s->a1, s->wf + bf_off(1), m + kOffB2, s->a2, nullptr,
                                                                train ? s->p2 : nullptr, nullptr, nwin);
  conv_kernel<kC, kC, EPI_HIDDEN, false><<<nwin, 128, 0, st>>>(s->a2, s->wf + bf_off(2), m + kOffB3, s->a3, nullptr,
                                                                train ? s->p3 : nullptr, nullptr, nwin);
  conv_kernel<kC, kCO, EPI_OUTPUT, false><<<nwin, 128, 0, st>>>(s->a3, s->wf + bf_off(3), m + kOffB4, nullptr, s->outf,
                                                                 nullptr, nullptr, nwin);
  return cudaGetLastError();
}

// gradients of the mean-square loss (outf vs tgt) into s->grad (overwritten, deterministic)
cudaError_t backward(rod_surrogate* s, int nwin, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(s->loss, 0, 4, st))) return e;
  const int64_t total = static_cast<int64_t>(nwin) * kRows * kCO;
  const float inv_count = 1.0f / (static_cast<float>(nwin) * kPos * kOut);
  loss_kernel<<<(total + 255) / 256, 256, 0, st>>>(s->outf, s->tgt, nwin, s->g4, s->loss, inv_count);
  const int wpb = kWgradWindows;
  const int gx = (nwin + wpb - 1) / wpb;
  float* gr = s->grad;
  auto reduce = [&](int n, float* dst) {
    reduce_partials_kernel<<<(n + 255) / 256, 256, 0, st>>>(s->part, gx, n, dst);
  };
  // layer 4: dW4, db4; input gradient to layer-3 activations (times SiLU'(p3))
  wgrad_kernel<kC, kCO><<<dim3(gx, (kTaps * kC + 63) / 64), 128, 0, st>>>(s->g4, s->a3, s->part, nwin, wpb);
  reduce(kW4 + kCO, gr + kOffW4);
  conv_kernel<kCO, kC, EPI_DGRAD, true><<<nwin, 128, 0, st>>>(s->g4, s->wt + bf_off(3), nullptr, s->g3, nullptr, nullptr,
                                                               s->p3, nwin);
  wgrad_kernel<kC, kC><<<dim3(gx, (kTaps * kC + 63) / 64), 128, 0, st>>>(s->g3, s->a2, s->part, nwin, wpb);
  reduce(kW3 + kC, gr + kOffW3);
  conv_kernel<kC, kC, EPI_DGRAD, true><<<nwin, 128, 0, st>>>(s->g3, s->wt + bf_off(2), nullptr, s->g2, nullptr, nullptr,
                                                              s->p2, nwin);
  wgrad_kernel<kC, kC><<<dim3(gx, (kTaps * kC + 63) / 64), 128, 0, st>>>(s->g2, s->a1, s->part, nwin, wpb);
  reduce(kW2 + kC, gr + kOffW2);
  conv_kernel<kC, kC, EPI_DGRAD, true><<<nwin, 128, 0, st>>>(s->g2, s->wt + bf_off(1), nullptr, s->g1, nullptr, nullptr,
                                                              s->p1, nwin);
  wgrad_kernel<kC0, kC><<<dim3(gx, (kTaps * kC0 + 63) / 64), 128, 0, st>>>(s->g1, s->a0, s->part, nwin, wpb);
  reduce(kW1 + kC, gr + kOffW1);
  return cudaGetLastError();
}

WinState win_state(const double* x, const double* v, const double* Q, const double* w, int nwin) {
  WinState S;
  S.x = x;
  S.v = v;
  S.Q = Q;
  S.w = w;
  S.N = static_cast<int64_t>(nwin) * kPos;
  S.E = static_cast<int64_t>(nwin) * (kPos - 1);
  return S;
}

}  // namespace

// accessors used by rod_api.cu to reach a system's state and constants
#include "rod_sysview.h"

namespace {

// After a synchronised call: ROD_ERR_TIMEOUT when a bounded wait of the fused kernel ran out
// (the system's error word; the step reports the word's other bits).
rod_status tc_wait_status(const SysView& V, const char* who) {
  int word = 0;
  cudaError_t e = cudaMemcpy(&word, V.err, sizeof word, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
  if (word & ERR_TIMEOUT) return internal_fail(ROD_ERR_TIMEOUT, who, "a bounded wait of the tensor-core kernel ran out");
  return ROD_OK;
}

rod_status check_system(rod_surrogate* s, rod_system* sys, SysView* V, const char* who) {
  rod_status rs = system_view(sys, V);
  if (rs != ROD_OK) return rs;
  if (V->max_n != kPos - 1 || V->min_n != kPos - 1)
    return internal_fail(ROD_ERR_ARG, who, "every rod must have 50 elements");
  if (V->contact) return internal_fail(ROD_ERR_ARG, who, "the surrogate advances rods without contact only");
  cudaError_t e;
  if ((e = grow(s, V->R)) || (e = refresh_weights(s, V->stream))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
  return ROD_OK;
}

// blocks of the fused kernel: one per SM (its shared memory holds the whole network)
cudaError_t fused_grid(int* grid) {
  static int sms = 0;
  static bool attr = false;
  cudaError_t e;
  if (!sms) {
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  }
  if (!attr) {
    if ((e = cudaFuncSetAttribute(tc_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem)))
      return e;
    attr = true;
  }
  *grid = sms;
  return cudaSuccess;
}

// n_calls network windows on the system's stream (no synchronisation): one fused launch per call
// (or the unfused kernel sequence when ROD_SURROGATE_UNFUSED is set, for comparison)
cudaError_t apply_calls(rod_surrogate* s, const SysView& V, int64_t n_calls, int reserve_sms = 0,
                        TcDebug dbg = TcDebug{nullptr, nullptr}) {
  const bool unfused = std::getenv("ROD_SURROGATE_UNFUSED") != nullptr;
  const WinState S = win_state(V.x, V.v, V.Q, V.w, V.R);
  int sms = 0;
  cudaError_t e;
  if (!unfused && (e = fused_grid(&sms))) return e;
  const int groups = (V.R + kGW - 1) / kGW;
  for (int64_t k = 0; k < n_calls; ++k) {
    if (unfused) {
      actuation_kernel<<<(V.R + 127) / 128, 128, 0, V.stream>>>(V.rods, V.R, *V.t, s->sc.T, s->act);
      features_kernel<<<V.R, kRows, 0, V.stream>>>(S, s->act, V.R, s->sc, s->a0);
      if ((e = forward(s, V.R, false, V.stream))) return e;
      apply_kernel<<<(V.R * kPos + 255) / 256, 256, 0, V.stream>>>(V.x, V.v, V.Q, V.w, V.N, V.E, V.R, s->outf, s->sc,
                                                                   V.rods);
    } else {
      const int grid = std::max(1, std::min((groups + kPipes - 1) / kPipes, sms - reserve_sms));
      tc_apply_kernel<<<grid, kTcThreads, kTcSmem, V.stream>>>(V.x, V.v, V.Q, V.w, V.N, V.E, V.R, V.rods, *V.t, s->sc,
                                                               s->wf, s->master, V.err,
                                                               s->wait_polls ? s->wait_polls : kWaitPolls, dbg);
      dbg = TcDebug{nullptr, nullptr};   // capture the first call only
    }
    *V.t += s->window * s->dt;
  }
  return cudaGetLastError();
}

// copy the system state to (to_ck = true) or from the checkpoint buffer on the system's stream
cudaError_t checkpoint(rod_surrogate* s, const SysView& V, bool to_ck) {
  const int64_t n = 6 * V.N + 12 * V.E;
  cudaError_t e;
  if (n > s->ck_cap) {
    if (s->ck) cudaFree(s->ck);
    s->ck = nullptr;
    s->ck_cap = 0;
    if ((e = cudaMalloc(&s->ck, n * 8))) return e;
    s->ck_cap = n;
  }
  double* parts[4] = {V.x, V.v, V.Q, V.w};
  const int64_t sizes[4] = {3 * V.N, 3 * V.N, 9 * V.E, 3 * V.E};
  int64_t off = 0;
  for (int k = 0; k < 4; ++k) {
    double* ck = s->ck + off;
    e = to_ck ? cudaMemcpyAsync(ck, parts[k], sizes[k] * 8, cudaMemcpyDeviceToDevice, V.stream)
              : cudaMemcpyAsync(parts[k], ck, sizes[k] * 8, cudaMemcpyDeviceToDevice, V.stream);
    if (e != cudaSuccess) return e;
    off += sizes[k];
  }
  return cudaSuccess;
}

// max relative tip error of the sampled rods of V against the rods of Ref (same order)
cudaError_t tip_error(rod_surrogate* s, const SysView& V, const SysView& Ref, int n_sample, double* out) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(s->err_dev, 0, sizeof(unsigned long long), V.stream))) return e;
  tip_error_kernel<<<1, 256, 0, V.stream>>>(V.x, V.N, Ref.x, Ref.N, s->sample, n_sample, V.rest_len, s->err_dev);
  if ((e = cudaMemcpyAsync(s->err_host, s->err_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost, V.stream)) ||
      (e = cudaStreamSynchronize(V.stream)))
    return e;
  uint64_t bits = *s->err_host;
  std::memcpy(out, &bits, 8);
  return cudaSuccess;
}

}  // namespace

extern "C" {

int64_t rod_surrogate_num_params(void) { return kNumParams; }

rod_status rod_surrogate_create(int32_t window_steps, double dt, rod_surrogate** out) {
  if (!out || window_steps < 1 || !(dt > 0) || !std::isfinite(dt))
    return internal_fail(ROD_ERR_ARG, "rod_surrogate_create: bad argument", "");
  rod_surrogate* s = new rod_surrogate();
  s->window = window_steps;
  s->dt = dt;
  s->sc.T = window_steps * dt;
  s->sc.prior_x = 1;
  s->sc.prior_q = 1;
  s->sc.keep_v = 1;
  s->sc.keep_w = 1;
  for (int c = 0; c < kFeat; ++c) {
    s->sc.in_shift[c] = 0.0;
    s->sc.in_shift_f[c] = 0.0f;
    s->sc.in_scale[c] = 1.0f;
  }
  for (int c = 0; c < kOut; ++c) s->sc.out[c] = 1.0;
  cudaError_t e;
  if ((e = cudaMalloc(&s->master, kNumParams * 4)) || (e = cudaMalloc(&s->grad, kNumParams * 4)) ||
      (e = cudaMalloc(&s->adam_m, kNumParams * 4)) || (e = cudaMalloc(&s->adam_v, kNumParams * 4)) ||
      (e = cudaMalloc(&s->wf, kBfTotal * 2)) || (e = cudaMalloc(&s->wt, kBfTotal * 2)) ||
      (e = cudaMalloc(&s->loss, 4)) || (e = cudaMalloc(&s->err_dev, 8)) ||
      (e = cudaMallocHost(&s->err_host, 8)) || (e = cudaMemset(s->master, 0, kNumParams * 4)) ||
      (e = cudaMemset(s->grad, 0, kNumParams * 4)) || (e = cudaMemset(s->adam_m, 0, kNumParams * 4)) ||
      (e = cudaMemset(s->adam_v, 0, kNumParams * 4))) {
    rod_surrogate_destroy(s);
    return internal_fail(ROD_ERR_CUDA, "rod_surrogate_create", cudaGetErrorString(e));
  }
  *out = s;
  return ROD_OK;
}

rod_status rod_surrogate_destroy(rod_surrogate* s) {
  if (!s) return ROD_OK;
  void* ptrs[] = {s->master, s->grad, s->adam_m, s->adam_v, s->wf, s->wt, s->loss, s->a0, s->a1, s->a2, s->a3,
                  s->p1, s->p2, s->p3, s->outf, s->tgt, s->g4, s->g3, s->g2, s->g1, s->act, s->ck, s->sample,
                  s->err_dev, s->part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->err_host) cudaFreeHost(s->err_host);
  for (auto& c : s->chk) {
    if (c.tips) cudaFree(c.tips);
    if (c.err_dev) cudaFree(c.err_dev);
    if (c.err_host) cudaFreeHost(c.err_host);
    if (c.gathered) cudaEventDestroy(c.gathered);
    if (c.tipped) cudaEventDestroy(c.tipped);
    if (c.done) cudaEventDestroy(c.done);
  }
  delete s;
  return ROD_OK;
}

rod_status rod_surrogate_set_params(rod_surrogate* s, const float* params, int on_device) {
  if (!s || !params) return internal_fail(ROD_ERR_ARG, "rod_surrogate_set_params: null argument", "");
  cudaError_t e = cudaMemcpy(s->master, params, kNumParams * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->adam_m, 0, kNumParams * 4);
  if (e == cudaSuccess) e = cudaMemset(s->adam_v, 0, kNumParams * 4);
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_set_params", cudaGetErrorString(e));
  s->adam_t = 0;
  s->weights_dirty = true;
  return ROD_OK;
}

rod_status rod_surrogate_get_params(rod_surrogate* s, float* params, int on_device) {
  if (!s || !params) return internal_fail(ROD_ERR_ARG, "rod_surrogate_get_params: null argument", "");
  cudaError_t e = cudaMemcpy(params, s->master, kNumParams * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_get_params", cudaGetErrorString(e));
  return ROD_OK;
}

rod_status rod_surrogate_set_scales(rod_surrogate* s, const double* in_shift, const double* in_scale,
                                    const double* out_scale) {
  if (!s || !in_shift || !in_scale || !out_scale)
    return internal_fail(ROD_ERR_ARG, "rod_surrogate_set_scales: null argument", "");
  for (int c = 0; c < kFeat; ++c)
    if (!std::isfinite(in_shift[c]) || !std::isfinite(in_scale[c]))
      return internal_fail(ROD_ERR_ARG, "rod_surrogate_set_scales: non-finite input scale", "");
  for (int c = 0; c < kOut; ++c)
    if (!(out_scale[c] > 0) || !std::isfinite(out_scale[c]))
      return internal_fail(ROD_ERR_ARG, "rod_surrogate_set_scales: output scales must be positive", "");
  for (int c = 0; c < kFeat; ++c) {
    s->sc.in_shift[c] = in_shift[c];
    s->sc.in_shift_f[c] = static_cast<float>(in_shift[c]);
    s->sc.in_scale[c] = static_cast<float>(in_scale[c]);
  }
  for (int c = 0; c < kOut; ++c) s->sc.out[c] = out_scale[c];
  return ROD_OK;
}

rod_status rod_surrogate_set_prior(rod_surrogate* s, int32_t flags) {
  if (!s || flags < 0 || flags > 15) return internal_fail(ROD_ERR_ARG, "rod_surrogate_set_prior: bad argument", "");
  s->sc.prior_x = flags & 1;
  s->sc.prior_q = (flags >> 1) & 1;
  s->sc.keep_v = !((flags >> 2) & 1);
  s->sc.keep_w = !((flags >> 3) & 1);
  return ROD_OK;
}

rod_status rod_surrogate_train_step(rod_surrogate* s, const double* x0, const double* v0, const double* Q0,
                                    const double* w0, const double* x1, const double* v1, const double* Q1,
                                    const double* w1, const double* act, int32_t nwin, float lr, float* loss_out,
                                    void* cuda_stream) {
  if (!s || !x0 || !v0 || !Q0 || !w0 || !x1 || !v1 || !Q1 || !w1 || !act || nwin < 1 || !std::isfinite(lr))
    return internal_fail(ROD_ERR_ARG, "rod_surrogate_train_step: bad argument", "");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e;
  if ((e = grow(s, nwin)) || (e = refresh_weights(s, st)))
    return internal_fail(ROD_ERR_CUDA, "rod_surrogate_train_step", cudaGetErrorString(e));
  const WinState A = win_state(x0, v0, Q0, w0, nwin), B = win_state(x1, v1, Q1, w1, nwin);
  features_kernel<<<nwin, kRows, 0, st>>>(A, act, nwin, s->sc, s->a0);
  targets_kernel<<<(static_cast<int64_t>(nwin) * kPos * kCO + 255) / 256, 256, 0, st>>>(A, B, nwin, s->sc, s->tgt);
  if ((e = forward(s, nwin, true, st)) || (e = backward(s, nwin, st)))
    return internal_fail(ROD_ERR_CUDA, "rod_surrogate_train_step", cudaGetErrorString(e));
  s->last_nwin = nwin;
  if (lr > 0.f) {
    s->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)s->adam_t), c2 = 1.f - powf(b2, (float)s->adam_t);
    adam_kernel<<<(kNumParams + 255) / 256, 256, 0, st>>>(s->master, s->grad, s->adam_m, s->adam_v, kNumParams, lr, b1,
                                                          b2, 1e-8f, c1, c2);
    s->weights_dirty = true;
  }
  if (loss_out) {
    if ((e = cudaMemcpyAsync(loss_out, s->loss, 4, cudaMemcpyDeviceToHost, st)) || (e = cudaStreamSynchronize(st)))
      return internal_fail(ROD_ERR_CUDA, "rod_surrogate_train_step", cudaGetErrorString(e));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_train_step", cudaGetErrorString(e));
  return ROD_OK;
}

rod_status rod_surrogate_get_grad(rod_surrogate* s, float* grad, int on_device) {
  if (!s || !grad) return internal_fail(ROD_ERR_ARG, "rod_surrogate_get_grad: null argument", "");
  cudaError_t e = cudaMemcpy(grad, s->grad, kNumParams * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_get_grad", cudaGetErrorString(e));
  return ROD_OK;
}

rod_status rod_surrogate_debug_buffer(rod_surrogate* s, int32_t which, float* out, int64_t cap, int64_t* n_out) {
  if (!s || !n_out || cap < 0 || (cap > 0 && !out))
    return internal_fail(ROD_ERR_ARG, "rod_surrogate_debug_buffer: bad argument", "");
  if (s->last_nwin < 1) return internal_fail(ROD_ERR_STATE, "rod_surrogate_debug_buffer: no training step yet", "");
  const int64_t nw = s->last_nwin, rows = nw * kRows;
  const void* src = nullptr;
  int64_t n = 0;
  bool bf = false;
  switch (which) {
    case 0: src = s->a0, n = rows * kC0, bf = true; break;
    case 1: src = s->a1, n = rows * kC, bf = true; break;
    case 2: src = s->a2, n = rows * kC, bf = true; break;
    case 3: src = s->a3, n = rows * kC, bf = true; break;
    case 4: src = s->p1, n = rows * kC; break;
    case 5: src = s->p2, n = rows * kC; break;
    case 6: src = s->p3, n = rows * kC; break;
    case 7: src = s->outf, n = nw * kPos * kCO; break;
    case 8: src = s->tgt, n = nw * kPos * kCO; break;
    case 9: src = s->g4, n = rows * kCO, bf = true; break;
    case 10: src = s->g3, n = rows * kC, bf = true; break;
    case 11: src = s->g2, n = rows * kC, bf = true; break;
    case 12: src = s->g1, n = rows * kC, bf = true; break;
    default: return internal_fail(ROD_ERR_ARG, "rod_surrogate_debug_buffer: which must be 0..12", "");
  }
  *n_out = n;
  if (cap == 0) return ROD_OK;
  if (cap < n) return internal_fail(ROD_ERR_ARG, "rod_surrogate_debug_buffer: buffer too small", "");
  cudaError_t e = cudaDeviceSynchronize();
  if (!e && !bf) e = cudaMemcpy(out, src, n * sizeof(float), cudaMemcpyDeviceToHost);
  if (!e && bf) {
    // BF16 bits widen to FP32 exactly: the 16 bits become the high half
    std::vector<uint16_t> h(static_cast<size_t>(n));
    e = cudaMemcpy(h.data(), src, n * sizeof(uint16_t), cudaMemcpyDeviceToHost);
    for (int64_t i = 0; !e && i < n; ++i) {
      const uint32_t u = static_cast<uint32_t>(h[i]) << 16;
      std::memcpy(out + i, &u, sizeof u);
    }
  }
  if (e) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_debug_buffer", cudaGetErrorString(e));
  return ROD_OK;
}

rod_status rod_surrogate_forward(rod_surrogate* s, const double* x, const double* v, const double* Q, const double* w,
                                 const double* act, int32_t nwin, float* out, void* cuda_stream) {
  if (!s || !x || !v || !Q || !w || !act || !out || nwin < 1)
    return internal_fail(ROD_ERR_ARG, "rod_surrogate_forward: bad argument", "");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e;
  if ((e = grow(s, nwin)) || (e = refresh_weights(s, st)))
    return internal_fail(ROD_ERR_CUDA, "rod_surrogate_forward", cudaGetErrorString(e));
  features_kernel<<<nwin, kRows, 0, st>>>(win_state(x, v, Q, w, nwin), act, nwin, s->sc, s->a0);
  if ((e = forward(s, nwin, false, st))) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_forward", cudaGetErrorString(e));
  e = cudaMemcpyAsync(out, s->outf, static_cast<size_t>(nwin) * kPos * kCO * 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_forward", cudaGetErrorString(e));
  return ROD_OK;
}

rod_status rod_surrogate_raw_features(rod_surrogate* s, const double* x, const double* v, const double* Q,
                                      const double* w, const double* act, int32_t nwin, double* out, int8_t* mask,
                                      void* cuda_stream) {
  if (!s || !x || !v || !Q || !w || !act || !out || nwin < 1)
    return internal_fail(ROD_ERR_ARG, "rod_surrogate_raw_features: bad argument", "");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int64_t n = static_cast<int64_t>(nwin) * kFeat * kPos;
  raw_features_kernel<<<(n + 255) / 256, 256, 0, st>>>(win_state(x, v, Q, w, nwin), act, nwin, out, mask);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_raw_features", cudaGetErrorString(e));
  return ROD_OK;
}

rod_status rod_surrogate_raw_targets(rod_surrogate* s, const double* x0, const double* v0, const double* Q0,
                                     const double* w0, const double* x1, const double* v1, const double* Q1,
                                     const double* w1, int32_t nwin, double* out, void* cuda_stream) {
  if (!s || !x0 || !v0 || !Q0 || !w0 || !x1 || !v1 || !Q1 || !w1 || !out || nwin < 1)
    return internal_fail(ROD_ERR_ARG, "rod_surrogate_raw_targets: bad argument", "");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int64_t n = static_cast<int64_t>(nwin) * kOut * kPos;
  raw_targets_kernel<<<(n + 255) / 256, 256, 0, st>>>(win_state(x0, v0, Q0, w0, nwin), win_state(x1, v1, Q1, w1, nwin),
                                                      nwin, s->sc.prior_x ? s->sc.T : 0.0,
                                                      s->sc.prior_q ? s->sc.T : 0.0, s->sc.keep_v, s->sc.keep_w, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_raw_targets", cudaGetErrorString(e));
  return ROD_OK;
}

rod_status rod_surrogate_perturb(rod_surrogate* s, const double* x0, const double* v0, const double* Q0,
                                 const double* w0, int32_t nwin, const double* rx, const double* rv, const double* rw,
                                 const double* ra, const double* spread, double noise, const int8_t* held, double* x,
                                 double* v, double* Q, double* w, void* cuda_stream) {
  const char* who = "rod_surrogate_perturb";
  if (!s || !x0 || !v0 || !Q0 || !w0 || nwin < 1 || !spread || !x || !v || !Q || !w || !(noise >= 0.0) ||
      (noise > 0.0 && (!rx || !rv || !rw || !ra)))
    return internal_fail(ROD_ERR_ARG, who, "bad argument");
  Spread sp{};
  sp.turn = 0.0;
  for (int c = 0; c < kOut; ++c) {
    if (!std::isfinite(spread[c])) return internal_fail(ROD_ERR_ARG, who, "non-finite spread");
    sp.s[c] = spread[c];
    if (c >= 6 && c < 12) sp.turn = std::max(sp.turn, spread[c]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int64_t n = static_cast<int64_t>(nwin) * kPos;
  perturb_kernel<<<(n + 255) / 256, 256, 0, st>>>(win_state(x0, v0, Q0, w0, nwin), nwin, rx, rv, rw, ra, sp, noise, held,
                                                  x, v, Q, w);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
  return ROD_OK;
}

rod_status rod_surrogate_apply(rod_surrogate* s, rod_system* sys, int64_t n_calls) {
  if (!s || !sys || n_calls < 0) return internal_fail(ROD_ERR_ARG, "rod_surrogate_apply: bad argument", "");
  SysView V;
  rod_status rs = check_system(s, sys, &V, "rod_surrogate_apply");
  if (rs != ROD_OK) return rs;
  cudaError_t e = apply_calls(s, V, n_calls);
  if (e == cudaSuccess) e = cudaStreamSynchronize(V.stream);
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_apply", cudaGetErrorString(e));
  return tc_wait_status(V, "rod_surrogate_apply");
}

rod_status rod_surrogate_set_wait_polls(rod_surrogate* s, uint32_t polls) {
  if (!s) return internal_fail(ROD_ERR_ARG, "rod_surrogate_set_wait_polls: null surrogate", "");
  s->wait_polls = polls;
  return ROD_OK;
}

rod_status rod_surrogate_apply_debug(rod_surrogate* s, rod_system* sys, float* pre, float* act, int64_t cap) {
  if (!s || !sys || !pre || !act) return internal_fail(ROD_ERR_ARG, "rod_surrogate_apply_debug: null argument", "");
  if (std::getenv("ROD_SURROGATE_UNFUSED"))
    return internal_fail(ROD_ERR_STATE, "rod_surrogate_apply_debug", "the capture needs the fused kernel");
  SysView V;
  rod_status rs = check_system(s, sys, &V, "rod_surrogate_apply_debug");
  if (rs != ROD_OK) return rs;
  const int64_t n = int64_t(4) * V.R * kPos * kC;
  if (cap < n) return internal_fail(ROD_ERR_ARG, "rod_surrogate_apply_debug", "buffers smaller than 4 x R x 51 x 64");
  // scratch of this debug call only
  float *dpre = nullptr, *dact = nullptr;
  cudaError_t e = cudaMalloc(&dpre, n * sizeof(float));
  if (!e) e = cudaMalloc(&dact, n * sizeof(float));
  if (!e) e = cudaMemsetAsync(dpre, 0, n * sizeof(float), V.stream);
  if (!e) e = cudaMemsetAsync(dact, 0, n * sizeof(float), V.stream);
  if (!e) e = apply_calls(s, V, 1, 0, TcDebug{dpre, dact});
  if (!e) e = cudaStreamSynchronize(V.stream);
  if (!e) e = cudaMemcpy(pre, dpre, n * sizeof(float), cudaMemcpyDeviceToHost);
  if (!e) e = cudaMemcpy(act, dact, n * sizeof(float), cudaMemcpyDeviceToHost);
  if (dpre) cudaFree(dpre);
  if (dact) cudaFree(dact);
  if (e != cudaSuccess) return internal_fail(ROD_ERR_CUDA, "rod_surrogate_apply_debug", cudaGetErrorString(e));
  return tc_wait_status(V, "rod_surrogate_apply_debug");
}

rod_status rod_surrogate_rollout(rod_surrogate* s, rod_system* sys, rod_system* shadow, const int32_t* sample_rods,
                                 int32_t n_sample, int64_t n_calls, int32_t check_every, double bound,
                                 rod_surrogate_stats* stats) {
  const char* who = "rod_surrogate_rollout";
  if (!s || !sys || !shadow || sys == shadow || !sample_rods || n_sample < 1 || n_calls < 0 || check_every < 1 ||
      !(bound > 0))
    return internal_fail(ROD_ERR_ARG, who, "bad argument");
  SysView V, H;
  rod_status rs = check_system(s, sys, &V, who);
  if (rs != ROD_OK) return rs;
  if ((rs = system_view(shadow, &H)) != ROD_OK) return rs;
  if (H.R != n_sample || H.max_n != kPos - 1 || H.min_n != kPos - 1 || H.contact)
    return internal_fail(ROD_ERR_ARG, who, "the shadow system must hold the n_sample rods (50 elements, no contact)");
  for (int i = 0; i < n_sample; ++i)
    if (sample_rods[i] < 0 || sample_rods[i] >= V.R) return internal_fail(ROD_ERR_ARG, who, "sample index out of range");
  if (std::fabs(*H.t - *V.t) > 1e-9 * std::max(1.0, std::fabs(*V.t)))
    return internal_fail(ROD_ERR_STATE, who, "the shadow system is not at the system's time");
  cudaError_t e;
  if (n_sample > s->sample_cap) {
    if (s->sample) cudaFree(s->sample);
    s->sample = nullptr;
    s->sample_cap = 0;
    if ((e = cudaMalloc(&s->sample, n_sample * 4))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
    s->sample_cap = n_sample;
  }
  if ((e = cudaMemcpyAsync(s->sample, sample_rods, n_sample * 4, cudaMemcpyHostToDevice, V.stream)))
    return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
  rod_surrogate_stats st{};
  for (int64_t done = 0; done < n_calls;) {
    const int64_t k = std::min<int64_t>(check_every, n_calls - done);
    const double t0 = *V.t;
    // the shadow rods follow the plain method on their own stream while the network runs
    if ((rs = rod_system_step_async(shadow, k * s->window, s->dt)) != ROD_OK) return rs;
    // the fused kernel fills a whole SM's shared memory: leave the shadow's blocks SMs of their own
    const int reserve = std::min(H.n_packs, 16);
    if ((e = checkpoint(s, V, true)) || (e = apply_calls(s, V, k, reserve)))
      return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
    if ((rs = rod_system_sync(shadow)) != ROD_OK) return rs;
    double err = 0.0;
    if ((e = tip_error(s, V, H, n_sample, &err))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
    st.checks += 1;
    if (err > bound) {
      // fall back: this segment again with the plain step from the checkpoint
      if ((e = checkpoint(s, V, false))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
      *V.t = t0;
      if ((rs = rod_system_step(sys, k * s->window, s->dt)) != ROD_OK) return rs;
      st.fallback_calls += k;
      st.rejected_err = std::max(st.rejected_err, err);
      if ((e = tip_error(s, V, H, n_sample, &err))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
    } else {
      st.surrogate_calls += k;
    }
    st.max_err = std::max(st.max_err, err);
    st.last_err = err;
    st.sum_err += err;
    done += k;
  }
  if (stats) *stats = st;
  return ROD_OK;
}

// Checked rollout with local (per-segment) error checks run in a pipeline: the check of a
// segment restarts the plain step from the surrogate's own state of the sampled rods at the
// segment's start, on a shadow system of its own, while the network goes on with the next
// segments; a segment whose local error exceeds the bound is undone (with everything after
// it) and redone with the plain step.
rod_status rod_surrogate_rollout_local(rod_surrogate* s, rod_system* sys, rod_system* const* shadows, int32_t n_shadows,
                                       const int32_t* sample_rods, int32_t n_sample, int64_t n_calls,
                                       int32_t check_every, double bound, rod_surrogate_stats* stats) {
  const char* who = "rod_surrogate_rollout_local";
  if (!s || !sys || !shadows || n_shadows < 1 || n_shadows > 8 || !sample_rods || n_sample < 1 || n_calls < 0 ||
      check_every < 1 || !(bound > 0))
    return internal_fail(ROD_ERR_ARG, who, "bad argument");
  SysView V;
  rod_status rs = check_system(s, sys, &V, who);
  if (rs != ROD_OK) return rs;
  std::vector<SysView> H(n_shadows);
  for (int k = 0; k < n_shadows; ++k) {
    if (!shadows[k] || shadows[k] == sys) return internal_fail(ROD_ERR_ARG, who, "bad shadow system");
    if ((rs = system_view(shadows[k], &H[k])) != ROD_OK) return rs;
    if (H[k].R != n_sample || H[k].max_n != kPos - 1 || H[k].min_n != kPos - 1 || H[k].contact)
      return internal_fail(ROD_ERR_ARG, who, "every shadow system must hold the n_sample rods (50 elements, no contact)");
    for (int q = 0; q < k; ++q)
      if (shadows[q] == shadows[k]) return internal_fail(ROD_ERR_ARG, who, "shadow systems must be distinct");
  }
  for (int i = 0; i < n_sample; ++i)
    if (sample_rods[i] < 0 || sample_rods[i] >= V.R) return internal_fail(ROD_ERR_ARG, who, "sample index out of range");
  cudaError_t e;
  const int64_t ss = 6 * V.N + 12 * V.E;  // one checkpoint
  const int slots = n_shadows;
  if (slots * ss > s->ck_cap) {
    if (s->ck) cudaFree(s->ck);
    s->ck = nullptr;
    s->ck_cap = 0;
    if ((e = cudaMalloc(&s->ck, slots * ss * 8))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
    s->ck_cap = slots * ss;
  }
  if (n_sample > s->sample_cap) {
    if (s->sample) cudaFree(s->sample);
    s->sample = nullptr;
    s->sample_cap = 0;
    if ((e = cudaMalloc(&s->sample, n_sample * 4))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
    s->sample_cap = n_sample;
  }
  // per slot: saved tips, error word (device and pinned host), events
  struct Slot {
    double* tips = nullptr;
    unsigned long long* err_dev = nullptr;
    unsigned long long* err_host = nullptr;
    cudaEvent_t gathered = nullptr, tipped = nullptr, done = nullptr;
    int64_t seg = -1;
    double t0 = 0.0;
  };
  std::vector<Slot> sl(slots);
  auto release = [&]() {
    for (auto& q : sl)
      if (q.done) cudaEventSynchronize(q.done);
  };
  auto failc = [&](cudaError_t err) {
    release();
    return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(err));
  };
  if (static_cast<int>(s->chk.size()) < slots) s->chk.resize(slots);
  for (int k = 0; k < slots; ++k) {
    rod_surrogate::CheckRes& c = s->chk[k];
    if (c.tips_cap < n_sample) {
      if (c.tips) cudaFree(c.tips);
      c.tips = nullptr;
      c.tips_cap = 0;
      if ((e = cudaMalloc(&c.tips, 3 * n_sample * 8))) return failc(e);
      c.tips_cap = n_sample;
    }
    if ((!c.err_dev && (e = cudaMalloc(&c.err_dev, 8))) || (!c.err_host && (e = cudaMallocHost(&c.err_host, 8))) ||
        (!c.gathered && (e = cudaEventCreateWithFlags(&c.gathered, cudaEventDisableTiming))) ||
        (!c.tipped && (e = cudaEventCreateWithFlags(&c.tipped, cudaEventDisableTiming))) ||
        (!c.done && (e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming))))
      return failc(e);
    sl[k].tips = c.tips;
    sl[k].err_dev = c.err_dev;
    sl[k].err_host = c.err_host;
    sl[k].gathered = c.gathered;
    sl[k].tipped = c.tipped;
    sl[k].done = c.done;
  }
  if ((e = cudaMemcpyAsync(s->sample, sample_rods, n_sample * 4, cudaMemcpyHostToDevice, V.stream))) return failc(e);
  int reserve = 0;
  for (int k = 0; k < n_shadows; ++k) reserve += H[k].n_packs;
  reserve = std::min(reserve, 64);
  // Segments: check_every calls each, except toward the end, where a segment has about a third
  // of the calls that follow it (at least one): a check runs its segment's plain steps after
  // the network has passed the segment's start, so the last checks end soon after the network
  // instead of a whole check_every-call check later.  A segment's allowance is its share of
  // the bound, bound x calls / check_every.
  std::vector<int64_t> seg_len;
  {
    int64_t after = 0;
    std::vector<int64_t> tail;
    while (after < n_calls) {
      int64_t L = std::max<int64_t>(1, std::min<int64_t>(check_every, after / 3));
      if (L == check_every) break;
      L = std::min(L, n_calls - after);
      tail.push_back(L);
      after += L;
    }
    const int64_t head = n_calls - after;   // covered by segments of check_every calls
    for (int64_t done = 0; done < head; done += check_every)
      seg_len.push_back(std::min<int64_t>(check_every, head - done));
    for (auto it = tail.rbegin(); it != tail.rend(); ++it) seg_len.push_back(*it);
  }
  std::vector<int64_t> seg_first(seg_len.size() + 1, 0);
  for (size_t k = 0; k < seg_len.size(); ++k) seg_first[k + 1] = seg_first[k] + seg_len[k];
  const int64_t n_seg = static_cast<int64_t>(seg_len.size());
  rod_surrogate_stats st{};
  int64_t seg = 0;
  int inflight = 0;
  // Wait for the check of slot q and act on it; returns true when the segment was rejected
  // (the system is then back at the segment's end, computed by the plain step).
  auto finish = [&](int qi, bool* rejected) -> rod_status {
    Slot& q = sl[qi];
    *rejected = false;
    if (q.seg < 0) return ROD_OK;
    if ((e = cudaEventSynchronize(q.done))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
    // a shadow that ran into non-finite values (from a non-finite surrogate state) fails the check
    rod_status r2 = rod_system_sync(shadows[qi]);
    if (r2 != ROD_OK && r2 != ROD_ERR_NONFINITE) return r2;
    double err;
    const uint64_t bits = *q.err_host;
    std::memcpy(&err, &bits, 8);
    if (r2 == ROD_ERR_NONFINITE) {
      err = INFINITY;
      if ((e = system_clear_error(shadows[qi]))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
    }
    const int64_t k = q.seg;
    const int64_t calls = seg_len[k];
    q.seg = -1;
    --inflight;
    st.checks += 1;
    st.last_err = err;
    if (err <= bound * static_cast<double>(calls) / check_every) {
      st.surrogate_calls += calls;
      st.max_err = std::max(st.max_err, err);
      st.sum_err += err;
      return ROD_OK;
    }
    // reject: drain the other checks (their segments come after this one and are discarded)
    for (int o = 0; o < slots; ++o)
      if (sl[o].seg >= 0) {
        if ((e = cudaEventSynchronize(sl[o].done))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
        r2 = rod_system_sync(shadows[o]);
        if (r2 == ROD_ERR_NONFINITE) {
          if ((e = system_clear_error(shadows[o]))) return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
        } else if (r2 != ROD_OK) {
          return r2;
        }
        sl[o].seg = -1;
        --inflight;
      }
    // back to the checkpoint of segment k and redo it with the plain step
    double* parts[4] = {V.x, V.v, V.Q, V.w};
    const int64_t sizes[4] = {3 * V.N, 3 * V.N, 9 * V.E, 3 * V.E};
    int64_t off = 0;
    for (int c = 0; c < 4; ++c) {
      if ((e = cudaMemcpyAsync(parts[c], s->ck + qi * ss + off, sizes[c] * 8, cudaMemcpyDeviceToDevice, V.stream)))
        return internal_fail(ROD_ERR_CUDA, who, cudaGetErrorString(e));
      off += sizes[c];
    }
    *V.t = q.t0;
    if ((r2 = rod_system_step(sys, calls * s->window, s->dt)) != ROD_OK) return r2;
    st.fallback_calls += calls;
    st.rejected_err = std::max(st.rejected_err, err);
    seg = k + 1;
    *rejected = true;
    return ROD_OK;
  };
  while (seg < n_seg || inflight > 0) {
    if (seg >= n_seg) {
      // drain the oldest check
      int oldest = -1;
      for (int q = 0; q < slots; ++q)
        if (sl[q].seg >= 0 && (oldest < 0 || sl[q].seg < sl[oldest].seg)) oldest = q;
      bool rej;
      rod_status r2 = finish(oldest, &rej);
      if (r2 != ROD_OK) {
        release();
        return r2;
      }
      continue;
    }
    const int qi = static_cast<int>(seg % slots);
    if (sl[qi].seg >= 0) {
      bool rej;
      rod_status r2 = finish(qi, &rej);
      if (r2 != ROD_OK) {
        release();
        return r2;
      }
      if (rej) continue;
    }
    Slot& q = sl[qi];
    const int64_t calls = seg_len[seg];
    q.seg = seg;
    q.t0 = *V.t;
    ++inflight;
    // checkpoint of the segment's start and the sampled rods' state into the slot's shadow
    {
      double* parts[4] = {V.x, V.v, V.Q, V.w};
      const int64_t sizes[4] = {3 * V.N, 3 * V.N, 9 * V.E, 3 * V.E};
      int64_t off = 0;
      for (int c = 0; c < 4; ++c) {
        if ((e = cudaMemcpyAsync(s->ck + qi * ss + off, parts[c], sizes[c] * 8, cudaMemcpyDeviceToDevice, V.stream)))
          return failc(e);
        off += sizes[c];
      }
    }
    gather_rods_kernel<<<(n_sample * kPos + 127) / 128, 128, 0, V.stream>>>(V.x, V.v, V.Q, V.w, V.N, V.E, s->sample,
                                                                           n_sample, H[qi].x, H[qi].v, H[qi].Q, H[qi].w);
    if ((e = cudaEventRecord(q.gathered, V.stream)) || (e = cudaStreamWaitEvent(H[qi].stream, q.gathered, 0)))
      return failc(e);
    rod_status r2 = rod_system_set_time(shadows[qi], q.t0);
    if (r2 == ROD_OK) r2 = rod_system_step_async(shadows[qi], calls * s->window, s->dt);
    if (r2 != ROD_OK) {
      release();
      return r2;
    }
    // the network's segment, then the sampled tips at its end
    if ((e = apply_calls(s, V, calls, reserve))) return failc(e);
    save_tips_kernel<<<(n_sample + 127) / 128, 128, 0, V.stream>>>(V.x, V.N, s->sample, n_sample, q.tips);
    if ((e = cudaEventRecord(q.tipped, V.stream)) || (e = cudaStreamWaitEvent(H[qi].stream, q.tipped, 0)) ||
        (e = cudaMemsetAsync(q.err_dev, 0, 8, H[qi].stream)))
      return failc(e);
    local_error_kernel<<<1, 256, 0, H[qi].stream>>>(H[qi].x, H[qi].N, q.tips, n_sample, H[qi].rest_len, q.err_dev);
    if ((e = cudaMemcpyAsync(q.err_host, q.err_dev, 8, cudaMemcpyDeviceToHost, H[qi].stream)) ||
        (e = cudaEventRecord(q.done, H[qi].stream)))
      return failc(e);
    ++seg;
  }
  if ((e = cudaStreamSynchronize(V.stream))) return failc(e);
  release();
  if (stats) *stats = st;
  return ROD_OK;
}

}  // extern "C"
