// rod_api.cu -- host side of librod: the C ABI declared in include/rod.h.
//
// The library owns its device memory (cudaMalloc at create, freed at destroy).  Everything
// that advances the state runs in the kernels of rod_step.cu and rod_contact.cu; the host
// only validates, derives per-rod constants once, packs rods into thread blocks and
// enqueues work on the system's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "../../include/rod.h"
#include "rod_adjoint.h"
#include "rod_contact.h"
#include "rod_diag.h"
#include "rod_internal.h"
#include "rod_sysview.h"

using namespace rod;

// ------------------------------------------------------------------------------ errors

static thread_local char g_msg[1024] = "";

static rod_status fail(rod_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof g_msg, fmt, ap);
  va_end(ap);
  return st;
}

namespace rod {
rod_status internal_fail(rod_status st, const char* what, const char* detail) {
  return fail(st, "%s%s%s", what, (detail && *detail) ? ": " : "", detail ? detail : "");
}
}  // namespace rod

#define CUDA_TRY(expr)                                                                               \
  do {                                                                                               \
    cudaError_t e_ = (expr);                                                                         \
    if (e_ != cudaSuccess) return fail(ROD_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------------------------ system

namespace {

constexpr int kMaxCapElems = 768;
constexpr double kPi = 3.14159265358979323846;

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t alloc(size_t count) {
    release();
    n = count;
    if (count == 0) return cudaSuccess;
    return cudaMalloc(&p, count * sizeof(T));
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

// Launch counter and optional CUDA-event timing of every kernel class.
struct Profiler {
  bool enabled = false;
  int64_t launches = 0;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t open_ev = nullptr;
  double total_ms[K_NUM_CLASSES] = {};
  int64_t count[K_NUM_CLASSES] = {};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  static void hook(void* ctx, int cls, int phase, cudaStream_t st) {
    Profiler* p = static_cast<Profiler*>(ctx);
    if (phase == 0) {
      p->launches += 1;
      if (p->enabled) {
        p->open_ev = p->get();
        cudaEventRecord(p->open_ev, st);
      }
    } else if (p->enabled && p->open_ev) {
      cudaEvent_t b = p->get();
      cudaEventRecord(b, st);
      p->pending.push_back(Rec{cls, p->open_ev, b});
      p->open_ev = nullptr;
    }
  }
  void collect() {
    for (auto& r : pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        total_ms[r.cls] += ms;
        count[r.cls] += 1;
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
  void reset() {
    collect();
    for (int k = 0; k < K_NUM_CLASSES; ++k) {
      total_ms[k] = 0.0;
      count[k] = 0;
    }
  }
  ~Profiler() {
    for (auto& r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

__global__ void set_time_kernel(double* t, double value) { *t = value; }
__global__ void advance_time_kernel(double* t, double dt) { *t += dt; }

__global__ void gather_clamp_kernel(const double* x, const double* Q, const RodConst* rods, int R, int64_t N, int64_t E,
                                    double* cx, double* cQ) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int j = rods[r].node0, i = rods[r].elem0;
  for (int c = 0; c < 3; ++c) cx[c * R + r] = x[c * N + j];
  for (int a = 0; a < 9; ++a) cQ[a * R + r] = Q[a * E + i];
}

// Non-finite values of a state array: the largest exponent field (all ones: Inf or NaN) on the
// integer pipe, one atomic per warp that saw one.
__global__ void nonfinite_kernel(const double* __restrict__ a, int64_t n, int* err) {
  unsigned mx = 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, static_cast<unsigned>(__double2hiint(a[i])) & 0x7FF00000u);
  if (__any_sync(0xffffffffu, mx == 0x7FF00000u) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_NONFINITE);
}

}  // namespace

// One captured CUDA graph of `steps` contact steps and what was baked into it.
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  int steps = 0;
  double dt = 0.0;
  int grid_version = -1;
  bool list = false;  // captured with the skin list
  int shape_version = -1;
  StepParams params{};  // the step kernel's parameters baked into the graph
};

struct rod_system {
  int R = 0;
  int64_t N = 0, E = 0, V = 0;
  int max_n = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // state
  DevBuf<double> x, v, Q, w;
  // constants
  DevBuf<double> rest_len, inv_rl, inv_rl2, inv_2D, sq_2D, Dhat, inv_m;
  DevBuf<double> rest_kappa, rest_sigma, elem_couple;
  DevBuf<double> magnet, arc0;  // magnetisation [3E], rest arc length of each element's first node [E]
  double field_b0[3] = {0, 0, 0}, field_bc[3] = {0, 0, 0}, field_bs[3] = {0, 0, 0}, field_omega = 0.0;
  int n_walls = 0;
  double wall_p[kMaxWalls][3] = {}, wall_n[kMaxWalls][3] = {}, wall_u[kMaxWalls][3] = {};
  double wall_k = 0.0, wall_c = 0.0, wall_mu = 0.0, wall_vslip = 0.0;
  DevBuf<double> clamp_x, clamp_Q;
  DevBuf<RodConst> rods;
  std::vector<RodConst> rods_h;
  std::vector<double> rest_len_h;
  // packing
  LaunchShape shape{0, 0, 0};
  DevBuf<Pack> packs;
  DevBuf<int2> pack_rods;  // (global rod, first pack-local element) of the rods of listed packs
  DevBuf<double> diag_rows, diag_tot;  // rod_system_diagnostics scratch: [9][R], [6]
  int n_packs = 0, n_listed = 0;
  // rods longer than a block holds: one pack each, run by cooperative launches with their
  // working arrays in long_scratch
  std::vector<Pack> long_packs;
  DevBuf<double> long_scratch;
  bool shape_user = false;
  // misc
  double gravity[3] = {0, 0, 0};
  bool has_gravity = false, has_act = false, has_damp_lin = false, has_damp_rot = false, has_tip = false;
  DevBuf<int> err;
  int* err_host = nullptr;  // pinned
  bool state_set = false;
  double t = 0.0;
  // contact
  ContactState contact;
  // launch accounting / timing
  Profiler prof;
  LaunchHook hook;
  // CUDA graphs of contact steps (captured on cap_stream, replayed on stream): one of
  // kGraphSteps steps for long calls and one of a single step for the rest of a call
  cudaStream_t cap_stream = nullptr;
  cudaStream_t body_stream = nullptr;  // captures the bodies of the graph's conditional nodes
  DevBuf<double> t_dev;
  StepGraph graphs[2];
  int shape_version = 0;
  bool use_graphs = true;
  // adjoint: checkpoints of the last checkpointed forward run, recompute buffers
  DevBuf<double> ckpt, seg_states, adj, final_state;
  int64_t ck_steps = 0, ck_every = 0;
  double ck_t0 = 0.0, ck_dt = 0.0;
  bool ck_valid = false;
  LaunchShape adj_shape{0, 0, 0};
  DevBuf<Pack> adj_packs;
  int adj_n_packs = 0;
};

namespace {

// Thread-block packs of an ensemble for one launch shape: rods longer than cap_elems get a
// cooperative pack each (longs); the others are packed consecutively in index order, or by
// best-fit decreasing when that needs fewer packs, whose packs then list their rods (global
// rod, first pack-local element) in list.  Host only; packs come heaviest first.
struct PackPlan {
  std::vector<Pack> packs, longs;
  std::vector<int2> list;
};

PackPlan plan_packs(const std::vector<RodConst>& rods, int cap_elems, int cap_rods) {
  PackPlan plan;
  std::vector<Pack>& packs = plan.packs;
  const int R = static_cast<int>(rods.size());
  Pack cur{};
  bool open = false;
  for (int r = 0; r < R; ++r) {
    const RodConst& rc = rods[r];
    const int n = rc.n;
    if (n > cap_elems) {
      // too long for a block: a pack of its own on the cooperative (grid-wide) path
      if (open) {
        packs.push_back(cur);
        open = false;
      }
      Pack lp{};
      lp.rod0 = r;
      lp.nrods = 1;
      lp.elem0 = rc.elem0;
      lp.nelem = n;
      lp.node0 = rc.node0;
      lp.nnode = n + 1;
      lp.vor0 = rc.elem0 - r;
      lp.nvor = n - 1;
      plan.longs.push_back(lp);
      continue;
    }
    if (open && (cur.nelem + n > cap_elems || cur.nrods + 1 > cap_rods)) {
      packs.push_back(cur);
      open = false;
    }
    if (!open) {
      cur = Pack{};
      cur.rod0 = r;
      cur.elem0 = rc.elem0;
      cur.node0 = rc.node0;
      cur.vor0 = rc.elem0 - r;
      open = true;
    }
    cur.nrods += 1;
    cur.nelem += n;
    cur.nnode += n + 1;
    cur.nvor += n - 1;
  }
  if (open) packs.push_back(cur);
  // Rods of mixed lengths leave the consecutive packs part empty (a block's element loops run
  // over cap_elems threads whatever the pack holds).  Best-fit decreasing over the same rods
  // fills them closer to the capacity; it is kept when it needs fewer packs.  It counts a rod's
  // nodes (n + 1), so a full pack's node loops make no second pass for a few nodes when the
  // block has as many threads as the capacity.  Its packs list their rods (global rod, first
  // pack-local element) unless the rods happen to be consecutive.
  {
    std::vector<int> order;
    for (int r = 0; r < R; ++r)
      if (rods[r].n <= cap_elems) order.push_back(r);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rods[a].n > rods[b].n; });
    std::vector<std::vector<int>> bins;
    std::vector<int> room;
    std::multiset<std::pair<int, int>> open_bins;  // (free node slots, bin), bins below cap_rods
    for (int r : order) {
      const int n = rods[r].n + 1;
      auto it = open_bins.lower_bound({n, -1});
      int b;
      if (it == open_bins.end()) {
        b = static_cast<int>(bins.size());
        bins.emplace_back();
        room.push_back(cap_elems);
      } else {
        b = it->second;
        open_bins.erase(it);
      }
      bins[b].push_back(r);
      room[b] -= n;
      if (static_cast<int>(bins[b].size()) < cap_rods) open_bins.insert({room[b], b});
    }
    if (bins.size() < packs.size()) {
      packs.clear();
      for (auto& bin : bins) {
        std::sort(bin.begin(), bin.end());
        Pack pk{};
        bool consecutive = true;
        for (size_t k = 1; k < bin.size(); ++k) consecutive = consecutive && bin[k] == bin[k - 1] + 1;
        const RodConst& first = rods[bin[0]];
        pk.rod0 = bin[0];
        pk.elem0 = first.elem0;
        pk.node0 = first.node0;
        pk.vor0 = first.elem0 - bin[0];
        pk.listed = consecutive ? 0 : 1;
        pk.list_off = consecutive ? 0 : static_cast<int32_t>(plan.list.size());
        for (int r : bin) {
          const int n = rods[r].n;
          if (!consecutive) plan.list.push_back(make_int2(r, pk.nelem));
          pk.nrods += 1;
          pk.nelem += n;
          pk.nnode += n + 1;
          pk.nvor += n - 1;
        }
        packs.push_back(pk);
      }
    }
  }
  // heaviest packs first (blocks start roughly in index order): the last, partly filled wave of
  // blocks then holds the lightest packs, which shortens the tail of every launch
  std::stable_sort(packs.begin(), packs.end(),
                   [](const Pack& a, const Pack& b) { return a.nelem + a.nnode > b.nelem + b.nnode; });
  return plan;
}

rod_status build_packs(rod_system* s, const LaunchShape& shape) {
  PackPlan plan = plan_packs(s->rods_h, shape.cap_elems, shape.cap_rods);
  const std::vector<Pack>& packs = plan.packs;
  const std::vector<int2>& list = plan.list;
  size_t scratch = 0;
  for (const Pack& lp : plan.longs) {
    LaunchShape ls;
    ls.cap_elems = lp.nelem;
    ls.cap_rods = 1;
    ls.threads = 256;
    scratch = std::max(scratch, step_smem_bytes(ls));
  }
  if (!list.empty()) {
    CUDA_TRY(s->pack_rods.alloc(list.size()));
    CUDA_TRY(cudaMemcpy(s->pack_rods.p, list.data(), list.size() * sizeof(int2), cudaMemcpyHostToDevice));
  } else {
    s->pack_rods.release();
  }
  if (!packs.empty()) {
    CUDA_TRY(s->packs.alloc(packs.size()));
    CUDA_TRY(cudaMemcpy(s->packs.p, packs.data(), packs.size() * sizeof(Pack), cudaMemcpyHostToDevice));
  }
  s->n_packs = static_cast<int>(packs.size());
  s->n_listed = static_cast<int>(std::count_if(packs.begin(), packs.end(), [](const Pack& p) { return p.listed != 0; }));
  s->long_packs = plan.longs;
  if (scratch > 0 && (int64_t)s->long_scratch.n * 8 < (int64_t)scratch)
    CUDA_TRY(s->long_scratch.alloc((scratch + 7) / 8));
  s->shape = shape;
  s->shape_version += 1;
  return ROD_OK;
}

// Rods per pack: as many of the shortest rods as the element capacity holds (at most 64), so
// the node arrays of a pack reserve no room a real pack cannot use.
int rods_per_pack(const rod_system* s, int cap_elems) {
  int min_n = 1 << 30;
  for (const auto& r : s->rods_h) min_n = std::min(min_n, r.n);
  if (s->rods_h.empty()) min_n = 1;
  return std::max(1, std::min(64, (cap_elems + min_n - 1) / min_n));
}

LaunchShape default_shape(const rod_system* s) {
  LaunchShape sh;
  int cap = 384;
  while (cap < s->max_n) cap += 128;
  sh.cap_elems = std::min(cap, kMaxCapElems);
  sh.cap_rods = rods_per_pack(s, sh.cap_elems);
  sh.threads = sh.cap_elems >= 512 ? 512 : 256;
  return sh;
}

StepParams make_params(rod_system* s) {
  StepParams P;
  std::memset(&P, 0, sizeof P);  // padding too: captured parameters are compared as whole objects
  P.x = s->x.p;
  P.v = s->v.p;
  P.Q = s->Q.p;
  P.w = s->w.p;
  P.N = s->N;
  P.E = s->E;
  P.V = s->V;
  P.rest_len = s->rest_len.p;
  P.inv_rl = s->inv_rl.p;
  P.inv_2D = s->inv_2D.p;
  P.sq_2D = s->sq_2D.p;
  P.Dhat = s->Dhat.p;
  P.inv_rl2 = s->inv_rl2.p;
  P.inv_m = s->inv_m.p;
  P.rest_kappa = s->rest_kappa.p;
  P.rest_sigma = s->rest_sigma.p;
  P.elem_couple = s->elem_couple.p;
  P.clamp_x = s->clamp_x.p;
  P.clamp_Q = s->clamp_Q.p;
  P.rods = s->rods.p;
  P.packs = s->packs.p;
  P.pack_rods = s->pack_rods.p;
  P.n_packs = s->n_packs;
  P.n_rods = s->R;
  for (int c = 0; c < 3; ++c) P.gravity[c] = s->gravity[c];
  P.has_gravity = s->has_gravity;
  P.has_damp_lin = s->has_damp_lin;
  P.has_damp_rot = s->has_damp_rot;
  P.has_tip = s->has_tip;
  P.has_act = s->has_act;
  P.magnet = s->magnet.p;
  for (int c = 0; c < 3; ++c) {
    P.field_b0[c] = s->field_b0[c];
    P.field_bc[c] = s->field_bc[c];
    P.field_bs[c] = s->field_bs[c];
  }
  P.field_omega = s->field_omega;
  P.arc0 = s->arc0.p;
  P.n_walls = s->n_walls;
  for (int k = 0; k < s->n_walls; ++k)
    for (int c = 0; c < 3; ++c) {
      P.wall_p[k][c] = s->wall_p[k][c];
      P.wall_n[k][c] = s->wall_n[k][c];
      P.wall_u[k][c] = s->wall_u[k][c];
    }
  P.wall_k = s->wall_k;
  P.wall_c = s->wall_c;
  P.wall_mu = s->wall_mu;
  P.wall_vslip = s->wall_vslip;
  P.fseg = nullptr;
  P.err = s->err.p;
  P.long_packs_h = s->long_packs.empty() ? nullptr : s->long_packs.data();
  P.n_long = static_cast<int32_t>(s->long_packs.size());
  P.long_scratch = s->long_scratch.p;
  return P;
}

rod_status read_error_word(rod_system* s) {
  CUDA_TRY(cudaMemcpyAsync(s->err_host, s->err.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  const int e = *s->err_host;
  if (e & ERR_NONFINITE) return fail(ROD_ERR_NONFINITE, "the state became non-finite (NaN/Inf)");
  if (e & ERR_GRID) return fail(ROD_ERR_OVERFLOW, "an element grew longer than the contact grid allows");
  if (e & ERR_OVERFLOW) return fail(ROD_ERR_OVERFLOW, "contact table capacity exceeded");
  if (e & ERR_TIMEOUT) return fail(ROD_ERR_TIMEOUT, "a bounded wait of the surrogate's tensor-core kernel ran out");
  return ROD_OK;
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

// Capture kGraphSteps contact steps (cell-list build, narrow phase, one step with binning of
// the next positions, time advance) once per (dt, launch shape, grid); replays then cost one
// launch per kGraphSteps steps.  The time of the state is read from t_dev inside the graph.
constexpr int kGraphSteps = 32;
// kernels per captured step: scan x3, fill, scatter, sort, records, gather, step, time; with the
// skin list decide, force, step, time, and the rebuild kernels (bin, scan x3, fill, scatter,
// sort, records, build, active set, snapshot) in a conditional node that the decision opens only when a
// rebuild is due (those launches are counted on the device)
constexpr int kKernelsPerGraphStep = 10;
constexpr int kKernelsPerListGraphStep = 4;

// One skin-list contact evaluation during the capture of s->cap_stream: the decision, an IF
// node whose body (captured on s->body_stream) holds the rebuild kernels, then the forces.
cudaError_t capture_list_step(rod_system* s) {
  LaunchHook none;
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s->cap_stream, &cst, nullptr, &g, &deps, nullptr, &nd);
  if (e) return e;
  if (cst != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle cond;
  if ((e = cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault))) return e;
  if ((e = contact_list_decide(s->contact, s->cap_stream, none, &cond))) return e;
  if ((e = cudaStreamGetCaptureInfo(s->cap_stream, &cst, nullptr, &g, &deps, nullptr, &nd))) return e;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp))) return e;
  if ((e = cudaStreamUpdateCaptureDependencies(s->cap_stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies)))
    return e;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(s->body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)))
    return e;
  e = contact_list_rebuild(s->contact, s->x.p, s->rods.p, s->N, s->E, s->err.p, s->body_stream, none);
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(s->body_stream, &out);
  if (e) return e;
  if (e2) return e2;
  return contact_list_force(s->contact, s->x.p, s->v.p, s->rods.p, s->N, s->E, s->err.p, s->cap_stream, none);
}

// The graph of g.steps contact steps for the current state, captured when something baked into
// it changed.  A capture that fails turns graphs off for the system (eager launches).
rod_status ensure_contact_graph(rod_system* s, StepGraph& g, const StepParams& Pb, double dt) {
  StepParams Pg = Pb;
  Pg.t_dev = s->t_dev.p;
  // reuse the graph while nothing baked into it has changed: the step kernel's parameters
  // (every pointer and constant; the structures are zero-initialised, so whole-object
  // comparison is exact), dt, the launch shape and the contact state's version
  const bool list = s->contact.skin > 0.0;
  if (g.exec && g.dt == dt && g.grid_version == s->contact.version && g.list == list &&
      g.shape_version == s->shape_version && std::memcmp(&g.params, &Pg, sizeof Pg) == 0)
    return ROD_OK;
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  LaunchHook none;
  cudaGraph_t graph = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < g.steps && e == cudaSuccess; ++k) {
    e = list ? capture_list_step(s)
             : contact_compute(s->contact, s->x.p, s->v.p, s->rods.p, s->N, s->E, s->R, s->err.p, s->cap_stream,
                               none, true);
    if (e == cudaSuccess) e = launch_pack_kernel(Pg, s->shape, MODE_ONE_STEP, 1, 0.0, dt, 0, nullptr, nullptr,
                                                 s->cap_stream, none);
    if (e == cudaSuccess) {
      advance_time_kernel<<<1, 1, 0, s->cap_stream>>>(s->t_dev.p, dt);
      e = cudaGetLastError();
    }
  }
  cudaError_t e2 = cudaStreamEndCapture(s->cap_stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    s->use_graphs = false;  // eager launches from now on
    return ROD_OK;
  }
  e = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g.exec = nullptr;
    cudaGetLastError();
    s->use_graphs = false;
    return ROD_OK;
  }
  g.dt = dt;
  g.grid_version = s->contact.version;
  g.list = list;
  g.shape_version = s->shape_version;
  g.params = Pg;
  return ROD_OK;
}

int64_t state_size(const rod_system* s) { return 6 * s->N + 12 * s->E; }

// copy the system state into / from one packed state [x v Q w]
cudaError_t pack_state(rod_system* s, double* dst) {
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dst, s->x.p, 3 * s->N * 8, cudaMemcpyDeviceToDevice, s->stream))) return e;
  if ((e = cudaMemcpyAsync(dst + 3 * s->N, s->v.p, 3 * s->N * 8, cudaMemcpyDeviceToDevice, s->stream))) return e;
  if ((e = cudaMemcpyAsync(dst + 6 * s->N, s->Q.p, 9 * s->E * 8, cudaMemcpyDeviceToDevice, s->stream))) return e;
  return cudaMemcpyAsync(dst + 6 * s->N + 9 * s->E, s->w.p, 3 * s->E * 8, cudaMemcpyDeviceToDevice, s->stream);
}
cudaError_t unpack_state(rod_system* s, const double* src) {
  cudaError_t e;
  if ((e = cudaMemcpyAsync(s->x.p, src, 3 * s->N * 8, cudaMemcpyDeviceToDevice, s->stream))) return e;
  if ((e = cudaMemcpyAsync(s->v.p, src + 3 * s->N, 3 * s->N * 8, cudaMemcpyDeviceToDevice, s->stream))) return e;
  if ((e = cudaMemcpyAsync(s->Q.p, src + 6 * s->N, 9 * s->E * 8, cudaMemcpyDeviceToDevice, s->stream))) return e;
  return cudaMemcpyAsync(s->w.p, src + 6 * s->N + 9 * s->E, 3 * s->E * 8, cudaMemcpyDeviceToDevice, s->stream);
}

// Launch shape of the adjoint kernel: the largest pack that fits the shared memory.
rod_status prepare_adjoint_shape(rod_system* s) {
  if (s->adj_n_packs) return ROD_OK;
  LaunchShape sh{0, 0, 256};
  for (int cap = 256; cap >= 32; cap -= 32) {
    sh.cap_elems = cap;
    sh.cap_rods = std::max(4, std::min(32, cap / 8));
    if (adjoint_smem_bytes(sh) <= 227 * 1024) break;
  }
  if (adjoint_smem_bytes(sh) > 227 * 1024 || sh.cap_elems < s->max_n)
    return fail(ROD_ERR_ARG, "the adjoint holds rods of at most %d elements in one thread block (longest rod: %d)",
                sh.cap_elems, s->max_n);
  std::vector<Pack> packs;
  Pack cur{};
  bool open = false;
  for (int r = 0; r < s->R; ++r) {
    const RodConst& rc = s->rods_h[r];
    if (open && (cur.nelem + rc.n > sh.cap_elems || cur.nrods + 1 > sh.cap_rods)) {
      packs.push_back(cur);
      open = false;
    }
    if (!open) {
      cur = Pack{};
      cur.rod0 = r;
      cur.elem0 = rc.elem0;
      cur.node0 = rc.node0;
      cur.vor0 = rc.elem0 - r;
      open = true;
    }
    cur.nrods += 1;
    cur.nelem += rc.n;
    cur.nnode += rc.n + 1;
    cur.nvor += rc.n - 1;
  }
  if (open) packs.push_back(cur);
  CUDA_TRY(s->adj_packs.alloc(packs.size()));
  CUDA_TRY(cudaMemcpy(s->adj_packs.p, packs.data(), packs.size() * sizeof(Pack), cudaMemcpyHostToDevice));
  s->adj_n_packs = static_cast<int>(packs.size());
  s->adj_shape = sh;
  return ROD_OK;
}

}  // namespace

// ------------------------------------------------------------------------------ ABI

extern "C" {

const char* rod_last_error(void) { return g_msg; }
const char* rod_version(void) { return "librod 1.0 (sm_103a, FP64)"; }
int32_t rod_max_elements_per_rod(void) { return kMaxCapElems; }

rod_status rod_system_create(const rod_system_desc* d, rod_system** out) {
  if (!d || !out) return fail(ROD_ERR_ARG, "null argument");
  *out = nullptr;
  if (d->n_rods <= 0) return fail(ROD_ERR_ARG, "n_rods must be positive (got %d)", d->n_rods);
  if (!d->n_elem || !d->rest_len || !d->radius || !d->youngs || !d->shear_mod || !d->density)
    return fail(ROD_ERR_ARG, "n_elem, rest_len, radius, youngs, shear_mod and density are required");
  const int R = d->n_rods;
  int64_t E = 0;
  int max_n = 0;
  for (int r = 0; r < R; ++r) {
    if (d->n_elem[r] < 1) return fail(ROD_ERR_ARG, "rod %d has %d elements (need >= 1)", r, d->n_elem[r]);
    E += d->n_elem[r];
    max_n = std::max(max_n, (int)d->n_elem[r]);
    if (!(d->radius[r] > 0) || !(d->youngs[r] > 0) || !(d->shear_mod[r] > 0) || !(d->density[r] > 0))
      return fail(ROD_ERR_ARG, "rod %d: radius, moduli and density must be positive and finite", r);
    if (!std::isfinite(d->radius[r]) || !std::isfinite(d->youngs[r]) || !std::isfinite(d->shear_mod[r]) ||
        !std::isfinite(d->density[r]))
      return fail(ROD_ERR_ARG, "rod %d: non-finite material parameter", r);
  }
  if (max_n > (1 << 24)) return fail(ROD_ERR_ARG, "a rod has %d elements (at most %d)", max_n, 1 << 24);
  if (E + R >= (int64_t(1) << 31) / 9) return fail(ROD_ERR_ARG, "ensemble too large (%lld elements)", (long long)E);
  for (int64_t i = 0; i < E; ++i)
    if (!(d->rest_len[i] > 0) || !std::isfinite(d->rest_len[i]))
      return fail(ROD_ERR_ARG, "rest length %lld must be positive and finite", (long long)i);
  if (!(d->alpha_c > 0) || !std::isfinite(d->alpha_c)) return fail(ROD_ERR_ARG, "alpha_c must be positive");
  if (!std::isfinite(d->nu_damp) || d->nu_damp < 0 || !std::isfinite(d->stokes_gamma) || d->stokes_gamma < 0)
    return fail(ROD_ERR_ARG, "nu_damp and stokes_gamma must be finite and >= 0");
  if (d->act_amp) {
    if (!d->act_period || !d->act_phase) return fail(ROD_ERR_ARG, "act_amp needs act_period and act_phase");
    for (int r = 0; r < R; ++r)
      if (!(d->act_period[r] > 0) || !std::isfinite(d->act_amp[r]) || !std::isfinite(d->act_phase[r]))
        return fail(ROD_ERR_ARG, "rod %d: actuation period must be positive, amplitude/phase finite", r);
  }
  const int64_t V = E - R, N = E + R;
  if (d->rest_kappa && !finite_all(d->rest_kappa, 3 * V)) return fail(ROD_ERR_ARG, "rest_kappa has non-finite values");
  if (d->rest_sigma && !finite_all(d->rest_sigma, 3 * E)) return fail(ROD_ERR_ARG, "rest_sigma has non-finite values");
  if (d->elem_couple && !finite_all(d->elem_couple, 3 * E)) return fail(ROD_ERR_ARG, "elem_couple has non-finite values");
  if (d->tip_force && !finite_all(d->tip_force, 3 * R)) return fail(ROD_ERR_ARG, "tip_force has non-finite values");
  for (int c = 0; c < 3; ++c)
    if (!std::isfinite(d->gravity[c])) return fail(ROD_ERR_ARG, "gravity must be finite");
  if (d->magnetization) {
    if (!finite_all(d->magnetization, 3 * E)) return fail(ROD_ERR_ARG, "magnetization has non-finite values");
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(d->field_b0[c]) || !std::isfinite(d->field_bc[c]) || !std::isfinite(d->field_bs[c]))
        return fail(ROD_ERR_ARG, "the magnetic field must be finite");
    if (!std::isfinite(d->field_omega)) return fail(ROD_ERR_ARG, "field_omega must be finite");
  }
  if (d->muscle_amp) {
    if (!d->muscle_period || !d->muscle_wavelength || !d->muscle_phase)
      return fail(ROD_ERR_ARG, "muscle_amp needs muscle_period, muscle_wavelength and muscle_phase");
    for (int r = 0; r < R; ++r)
      if (!std::isfinite(d->muscle_amp[r]) || !(d->muscle_period[r] > 0) || !(d->muscle_wavelength[r] > 0) ||
          !std::isfinite(d->muscle_period[r]) || !std::isfinite(d->muscle_wavelength[r]) ||
          !std::isfinite(d->muscle_phase[r]))
        return fail(ROD_ERR_ARG, "rod %d: muscle period and wavelength must be positive, amplitude/phase finite", r);
  }
  if (d->n_walls < 0 || d->n_walls > kMaxWalls) return fail(ROD_ERR_ARG, "n_walls must be 0..%d", kMaxWalls);
  if (d->n_walls > 0) {
    if (!d->wall_point || !d->wall_normal) return fail(ROD_ERR_ARG, "walls need wall_point and wall_normal");
    for (int k = 0; k < d->n_walls; ++k) {
      const double* nn = d->wall_normal + 3 * k;
      if (!finite_all(d->wall_point + 3 * k, 3) || !finite_all(nn, 3) ||
          (d->wall_velocity && !finite_all(d->wall_velocity + 3 * k, 3)))
        return fail(ROD_ERR_ARG, "wall %d: non-finite point, normal or velocity", k);
      if (std::fabs(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2] - 1.0) > 1e-12)
        return fail(ROD_ERR_ARG, "wall %d: the normal must be a unit vector", k);
    }
    if (!(d->wall_k >= 0) || !(d->wall_c >= 0) || !(d->wall_mu >= 0) || !std::isfinite(d->wall_k) ||
        !std::isfinite(d->wall_c) || !std::isfinite(d->wall_mu) || (d->wall_mu > 0 && !(d->wall_vslip > 0)))
      return fail(ROD_ERR_ARG, "walls need k, c, mu >= 0 and, with friction, a positive slip velocity");
  }

  rod_system* s = new rod_system();
  s->hook.fn = &Profiler::hook;
  s->hook.ctx = &s->prof;
  s->R = R;
  s->E = E;
  s->N = N;
  s->V = V;
  s->max_n = max_n;
  auto cleanup = [&](rod_status st) {
    rod_system_destroy(s);
    return st;
  };
  if (d->cuda_stream) {
    s->stream = static_cast<cudaStream_t>(d->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(fail(ROD_ERR_CUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(cudaGetLastError())));
    s->own_stream = true;
  }

  // per-rod constants
  s->rods_h.resize(R);
  int64_t e0 = 0, n0 = 0;
  bool any_act = false;
  for (int r = 0; r < R; ++r) {
    RodConst& rc = s->rods_h[r];
    std::memset(&rc, 0, sizeof rc);
    const double rad = d->radius[r], Ey = d->youngs[r], G = d->shear_mod[r], rho = d->density[r];
    const double A = kPi * rad * rad;
    const double I1 = kPi * rad * rad * rad * rad / 4.0;
    const double I[3] = {I1, I1, 2.0 * I1};
    rc.S[0] = d->alpha_c * G * A;
    rc.S[1] = d->alpha_c * G * A;
    rc.S[2] = Ey * A;
    rc.B[0] = Ey * I[0];
    rc.B[1] = Ey * I[1];
    rc.B[2] = G * I[2];
    for (int c = 0; c < 3; ++c) {
      rc.rhoI[c] = rho * I[c];
      rc.inv_rhoI[c] = 1.0 / (rho * I[c]);
    }
    rc.damp_lin = (d->nu_damp + d->stokes_gamma) / (rho * A);
    rc.damp_rot = d->nu_damp / (rho * A);
    s->has_damp_lin = s->has_damp_lin || rc.damp_lin != 0.0;
    s->has_damp_rot = s->has_damp_rot || rc.damp_rot != 0.0;
    rc.rhoI_12 = rc.rhoI[1] - rc.rhoI[2];
    rc.B_21 = rc.B[2] - rc.B[1];
    rc.B_21q = 0.25 * rc.B_21;
    rc.radius = rad;
    rc.radius_f = static_cast<float>(rad);
    rc.node0 = static_cast<int32_t>(n0);
    rc.elem0 = static_cast<int32_t>(e0);
    rc.n = d->n_elem[r];
    rc.clamp = (d->clamp_base && d->clamp_base[r]) ? 1 : 0;
    rc.act_elem = -1;
    if (d->act_amp && d->act_amp[r] != 0.0) {
      rc.act_amp = d->act_amp[r];
      rc.act_omega = 2.0 * kPi / d->act_period[r];
      rc.act_phase = d->act_phase[r];
      rc.act_elem = (rc.clamp && rc.n >= 2) ? 1 : 0;
      any_act = true;
    }
    if (d->tip_force)
      for (int c = 0; c < 3; ++c) {
        rc.tip[c] = d->tip_force[c * R + r];
        s->has_tip = s->has_tip || rc.tip[c] != 0.0;
      }
    if (d->muscle_amp && d->muscle_amp[r] != 0.0) {
      rc.muscle_amp = d->muscle_amp[r];
      rc.muscle_omega = 2.0 * kPi / d->muscle_period[r];
      rc.muscle_k = 2.0 * kPi / d->muscle_wavelength[r];
      rc.muscle_phase = d->muscle_phase[r];
    }
    e0 += rc.n;
    n0 += rc.n + 1;
  }
  s->has_act = any_act;
  for (int c = 0; c < 3; ++c) {
    s->gravity[c] = d->gravity[c];
    if (d->magnetization) {
      s->field_b0[c] = d->field_b0[c];
      s->field_bc[c] = d->field_bc[c];
      s->field_bs[c] = d->field_bs[c];
    }
  }
  s->field_omega = d->magnetization ? d->field_omega : 0.0;
  s->n_walls = d->n_walls;
  for (int k = 0; k < d->n_walls; ++k)
    for (int c = 0; c < 3; ++c) {
      s->wall_p[k][c] = d->wall_point[3 * k + c];
      s->wall_n[k][c] = d->wall_normal[3 * k + c];
      s->wall_u[k][c] = d->wall_velocity ? d->wall_velocity[3 * k + c] : 0.0;
    }
  s->wall_k = d->wall_k;
  s->wall_c = d->wall_c;
  s->wall_mu = d->wall_mu;
  s->wall_vslip = d->wall_vslip;
  s->has_gravity = d->gravity[0] != 0.0 || d->gravity[1] != 0.0 || d->gravity[2] != 0.0;

  // per-item constants
  s->rest_len_h.assign(d->rest_len, d->rest_len + E);
  std::vector<double> inv_rl(E), inv_rl2(E), inv_2D(std::max<int64_t>(V, 1)), sq_2D(std::max<int64_t>(V, 1)),
      Dh(std::max<int64_t>(V, 1)), inv_m(N);
  for (int r = 0; r < R; ++r) {
    const RodConst& rc = s->rods_h[r];
    const double rhoA = d->density[r] * kPi * d->radius[r] * d->radius[r];
    for (int i = 0; i < rc.n; ++i) {
      inv_rl[rc.elem0 + i] = 1.0 / d->rest_len[rc.elem0 + i];
      inv_rl2[rc.elem0 + i] = inv_rl[rc.elem0 + i] * inv_rl[rc.elem0 + i];
    }
    for (int k = 0; k < rc.n - 1; ++k) {
      const double a = d->rest_len[rc.elem0 + k], b = d->rest_len[rc.elem0 + k + 1];
      inv_2D[rc.elem0 - r + k] = 1.0 / (a + b);
      sq_2D[rc.elem0 - r + k] = (a + b) * (a + b);
      Dh[rc.elem0 - r + k] = 0.5 * (a + b);
    }
    for (int j = 0; j <= rc.n; ++j) {
      const double left = j >= 1 ? d->rest_len[rc.elem0 + j - 1] : 0.0;
      const double right = j < rc.n ? d->rest_len[rc.elem0 + j] : 0.0;
      inv_m[rc.node0 + j] = 1.0 / (0.5 * rhoA * (left + right));
    }
  }

  auto up = [&](auto& buf, const auto* src, size_t count) -> cudaError_t {
    cudaError_t e = buf.alloc(count);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(buf.p, src, count * sizeof(*src), cudaMemcpyHostToDevice);
  };
  cudaError_t ce = cudaSuccess;
  if ((ce = s->x.alloc(3 * N)) || (ce = s->v.alloc(3 * N)) || (ce = s->Q.alloc(9 * E)) || (ce = s->w.alloc(3 * E)) ||
      (ce = up(s->rest_len, d->rest_len, E)) || (ce = up(s->inv_rl, inv_rl.data(), E)) ||
      (ce = up(s->inv_rl2, inv_rl2.data(), E)) ||
      (ce = up(s->inv_2D, inv_2D.data(), inv_2D.size())) || (ce = up(s->sq_2D, sq_2D.data(), sq_2D.size())) ||
      (ce = up(s->Dhat, Dh.data(), Dh.size())) ||
      (ce = up(s->inv_m, inv_m.data(), N)) || (ce = up(s->rods, s->rods_h.data(), R)) ||
      (ce = s->clamp_x.alloc(3 * R)) || (ce = s->clamp_Q.alloc(9 * R)) || (ce = s->err.alloc(1)))
    return cleanup(fail(ROD_ERR_CUDA, "device allocation/copy failed: %s", cudaGetErrorString(ce)));
  if (d->rest_kappa && V > 0 && (ce = up(s->rest_kappa, d->rest_kappa, 3 * V)))
    return cleanup(fail(ROD_ERR_CUDA, "copy failed: %s", cudaGetErrorString(ce)));
  if (d->rest_sigma && (ce = up(s->rest_sigma, d->rest_sigma, 3 * E)))
    return cleanup(fail(ROD_ERR_CUDA, "copy failed: %s", cudaGetErrorString(ce)));
  if (d->elem_couple && (ce = up(s->elem_couple, d->elem_couple, 3 * E)))
    return cleanup(fail(ROD_ERR_CUDA, "copy failed: %s", cudaGetErrorString(ce)));
  if (d->magnetization && (ce = up(s->magnet, d->magnetization, 3 * E)))
    return cleanup(fail(ROD_ERR_CUDA, "copy failed: %s", cudaGetErrorString(ce)));
  bool any_muscle = false;
  for (int r = 0; r < R; ++r) any_muscle = any_muscle || s->rods_h[r].muscle_amp != 0.0;
  if (any_muscle) {
    // rest arc length of every element's first node, summed along each rod in order
    std::vector<double> arc(E);
    for (int r = 0; r < R; ++r) {
      double acc = 0.0;
      for (int i = 0; i < s->rods_h[r].n; ++i) {
        arc[s->rods_h[r].elem0 + i] = acc;
        acc += d->rest_len[s->rods_h[r].elem0 + i];
      }
    }
    if ((ce = up(s->arc0, arc.data(), E))) return cleanup(fail(ROD_ERR_CUDA, "copy failed: %s", cudaGetErrorString(ce)));
  }
  if ((ce = s->t_dev.alloc(1)) || (ce = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking)) ||
      (ce = cudaStreamCreateWithFlags(&s->body_stream, cudaStreamNonBlocking)))
    return cleanup(fail(ROD_ERR_CUDA, "allocation failed: %s", cudaGetErrorString(ce)));
  if ((ce = cudaMemset(s->err.p, 0, sizeof(int))) || (ce = cudaMallocHost(&s->err_host, sizeof(int))))
    return cleanup(fail(ROD_ERR_CUDA, "allocation failed: %s", cudaGetErrorString(ce)));
  *s->err_host = 0;
  s->graphs[0].steps = kGraphSteps;
  s->graphs[1].steps = 1;
  rod_status st = build_packs(s, default_shape(s));
  if (st != ROD_OK) return cleanup(st);
  *out = s;
  return ROD_OK;
}

rod_status rod_system_destroy(rod_system* s) {
  if (!s) return ROD_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  s->x.release();
  s->v.release();
  s->Q.release();
  s->w.release();
  s->rest_len.release();
  s->inv_rl.release();
  s->inv_2D.release();
  s->sq_2D.release();
  s->Dhat.release();
  s->inv_rl2.release();
  s->inv_m.release();
  s->rest_kappa.release();
  s->rest_sigma.release();
  s->elem_couple.release();
  s->magnet.release();
  s->arc0.release();
  s->clamp_x.release();
  s->clamp_Q.release();
  s->rods.release();
  s->packs.release();
  s->pack_rods.release();
  s->diag_rows.release();
  s->diag_tot.release();
  s->long_scratch.release();
  s->ckpt.release();
  s->seg_states.release();
  s->adj.release();
  s->final_state.release();
  s->adj_packs.release();
  s->err.release();
  contact_release(s->contact);
  for (StepGraph& g : s->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->body_stream) cudaStreamDestroy(s->body_stream);
  s->t_dev.release();
  if (s->err_host) cudaFreeHost(s->err_host);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return ROD_OK;
}

rod_status rod_system_sizes(const rod_system* s, int64_t* n_nodes, int64_t* n_elems, int64_t* n_voronoi) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (n_nodes) *n_nodes = s->N;
  if (n_elems) *n_elems = s->E;
  if (n_voronoi) *n_voronoi = s->V;
  return ROD_OK;
}

rod_status rod_system_set_state(rod_system* s, const double* x, const double* v, const double* Q, const double* w,
                                int on_device) {
  if (!s || !x || !v || !Q || !w) return fail(ROD_ERR_ARG, "null argument");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(cudaMemcpyAsync(s->x.p, x, 3 * s->N * sizeof(double), kind, s->stream));
  CUDA_TRY(cudaMemcpyAsync(s->v.p, v, 3 * s->N * sizeof(double), kind, s->stream));
  CUDA_TRY(cudaMemcpyAsync(s->Q.p, Q, 9 * s->E * sizeof(double), kind, s->stream));
  CUDA_TRY(cudaMemcpyAsync(s->w.p, w, 3 * s->E * sizeof(double), kind, s->stream));
  if (!on_device) {
    // host input: checked for non-finite values on the device after the copy (the copy of a
    // host state has to synchronise anyway); a rejected state leaves the system without one
    CUDA_TRY(cudaMemsetAsync(s->err.p, 0, sizeof(int), s->stream));
    const struct { const double* p; int64_t n; } arr[4] = {{s->x.p, 3 * s->N}, {s->v.p, 3 * s->N},
                                                           {s->Q.p, 9 * s->E}, {s->w.p, 3 * s->E}};
    for (const auto& a : arr) {
      const int64_t blocks = std::min<int64_t>((a.n + 255) / 256, 4096);
      s->hook.before(K_MISC, s->stream);
      nonfinite_kernel<<<static_cast<unsigned>(std::max<int64_t>(blocks, 1)), 256, 0, s->stream>>>(a.p, a.n, s->err.p);
      s->hook.after(K_MISC, s->stream);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(s->err_host, s->err.p, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (*s->err_host != 0) {
      s->state_set = false;
      CUDA_TRY(cudaMemsetAsync(s->err.p, 0, sizeof(int), s->stream));
      CUDA_TRY(cudaStreamSynchronize(s->stream));
      return fail(ROD_ERR_ARG, "the state holds non-finite values");
    }
  }
  s->hook.before(K_MISC, s->stream);
  gather_clamp_kernel<<<(s->R + 127) / 128, 128, 0, s->stream>>>(s->x.p, s->Q.p, s->rods.p, s->R, s->N, s->E,
                                                                  s->clamp_x.p, s->clamp_Q.p);
  s->hook.after(K_MISC, s->stream);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemsetAsync(s->err.p, 0, sizeof(int), s->stream));
  if (!on_device) CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->state_set = true;
  s->t = 0.0;
  s->contact.grid_valid = false;
  return ROD_OK;
}

rod_status rod_system_get_state(rod_system* s, double* x, double* v, double* Q, double* w, int on_device) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (!s->state_set) return fail(ROD_ERR_STATE, "no state has been set");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (x) CUDA_TRY(cudaMemcpyAsync(x, s->x.p, 3 * s->N * sizeof(double), kind, s->stream));
  if (v) CUDA_TRY(cudaMemcpyAsync(v, s->v.p, 3 * s->N * sizeof(double), kind, s->stream));
  if (Q) CUDA_TRY(cudaMemcpyAsync(Q, s->Q.p, 9 * s->E * sizeof(double), kind, s->stream));
  if (w) CUDA_TRY(cudaMemcpyAsync(w, s->w.p, 3 * s->E * sizeof(double), kind, s->stream));
  if (!on_device) CUDA_TRY(cudaStreamSynchronize(s->stream));
  return ROD_OK;
}

rod_status rod_system_set_time(rod_system* s, double t) {
  if (!s || !std::isfinite(t)) return fail(ROD_ERR_ARG, "bad argument");
  s->t = t;
  return ROD_OK;
}

rod_status rod_system_get_time(const rod_system* s, double* t) {
  if (!s || !t) return fail(ROD_ERR_ARG, "null argument");
  *t = s->t;
  return ROD_OK;
}

rod_status rod_system_step_async(rod_system* s, int64_t n_steps, double dt) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (!s->state_set) return fail(ROD_ERR_STATE, "no state has been set");
  if (n_steps < 0 || !(dt > 0) || !std::isfinite(dt)) return fail(ROD_ERR_ARG, "need n_steps >= 0 and dt > 0");
  if (n_steps == 0) return ROD_OK;
  StepParams P = make_params(s);
  if (!s->contact.enabled) {
    const int64_t chunk = int64_t(1) << 20;
    for (int64_t done = 0; done < n_steps; done += chunk) {
      const int64_t k = std::min(chunk, n_steps - done);
      CUDA_TRY(launch_pack_kernel(P, s->shape, MODE_STEPS, k, s->t + done * dt, dt, 1, nullptr, nullptr, s->stream, s->hook));
    }
  } else {
    rod_status st = contact_prepare(s->contact, s->rods_h, s->rods.p, s->x.p, s->N, s->E, s->R, s->stream, s->hook);
    if (st != ROD_OK) return st;
    P.fseg = s->contact.fseg;
    const bool list = s->contact.skin > 0.0;
    StepParams Pb = P;  // with the binning epilogue for the next step, or the skin list's displacement
    if (list) {
      contact_list_params(s->contact, P);
      Pb = P;
    } else {
      contact_bin_params(s->contact, Pb);
    }
    CUDA_TRY(contact_clear_counts(s->contact, s->stream));
    CUDA_TRY(launch_pack_kernel(Pb, s->shape, MODE_KIN_HALF, 1, s->t, dt, 0, nullptr, nullptr, s->stream, s->hook));
    // steps 0 .. n-2 bin the next step's positions; the last one ends on a half step
    const int64_t binned = n_steps - 1;
    int64_t k = 0;
    // Binned steps replay the kGraphSteps-step graph, then the one-step graph for the rest.
    // (cooperative launches of long rods stay eager: no graph replay when there are any)
    if (s->use_graphs && !s->prof.enabled && binned >= 1 && s->long_packs.empty()) {
      bool time_set = false;
      for (StepGraph& g : s->graphs) {
        if (binned - k < g.steps) continue;
        st = ensure_contact_graph(s, g, Pb, dt);
        if (st != ROD_OK) return st;
        if (!g.exec) break;
        if (!time_set) {
          set_time_kernel<<<1, 1, 0, s->stream>>>(s->t_dev.p, s->t);
          CUDA_TRY(cudaGetLastError());
          s->prof.launches += 1;
          time_set = true;
        }
        for (; k + g.steps <= binned; k += g.steps) {
          CUDA_TRY(cudaGraphLaunch(g.exec, s->stream));
          s->prof.launches += g.steps * (list ? kKernelsPerListGraphStep : kKernelsPerGraphStep);
        }
      }
    }
    for (; k < n_steps; ++k) {
      const bool last = (k == n_steps - 1);
      if (list)
        CUDA_TRY(contact_list_compute(s->contact, s->x.p, s->v.p, s->rods.p, s->N, s->E, s->R, s->err.p, s->stream,
                                      s->hook));
      else
        CUDA_TRY(contact_compute(s->contact, s->x.p, s->v.p, s->rods.p, s->N, s->E, s->R, s->err.p, s->stream,
                                 s->hook, true));
      CUDA_TRY(launch_pack_kernel(last ? P : Pb, s->shape, MODE_ONE_STEP, 1, s->t + k * dt, dt, last ? 1 : 0, nullptr,
                                  nullptr, s->stream, s->hook));
    }
  }
  s->t += n_steps * dt;
  return ROD_OK;
}

rod_status rod_system_sync(rod_system* s) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  return read_error_word(s);
}

rod_status rod_system_step(rod_system* s, int64_t n_steps, double dt) {
  rod_status st = rod_system_step_async(s, n_steps, dt);
  if (st != ROD_OK) return st;
  return read_error_word(s);
}

rod_status rod_system_contact_config(rod_system* s, int enable, double k, double c, double cell_size) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (enable && (!(k >= 0) || !(c >= 0) || !std::isfinite(k) || !std::isfinite(c) || !std::isfinite(cell_size)))
    return fail(ROD_ERR_ARG, "contact needs finite k >= 0, c >= 0 and cell_size");
  s->contact.enabled = enable != 0;
  s->contact.k = k;
  s->contact.c = c;
  s->contact.cell_size = cell_size;
  s->contact.grid_valid = false;
  return ROD_OK;
}

rod_status rod_system_contact_skin(rod_system* s, double skin) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (!(skin >= 0) || !std::isfinite(skin)) return fail(ROD_ERR_ARG, "the skin must be finite and >= 0");
  s->contact.skin = skin;
  s->contact.grid_valid = false;  // the cell edge covers the skin
  return ROD_OK;
}

rod_status rod_system_contact_list_builds(rod_system* s, int64_t* n) {
  if (!s || !n) return fail(ROD_ERR_ARG, "null argument");
  *n = 0;
  if (!s->contact.ctl || !(s->contact.skin > 0.0) || !s->contact.grid_valid) return ROD_OK;
  ListCtl c{};
  CUDA_TRY(cudaMemcpyAsync(&c, s->contact.ctl, sizeof(ListCtl), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  *n = c.builds;
  return ROD_OK;
}

rod_status rod_system_friction(rod_system* s, double mu, double v_slip) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (!(mu >= 0) || !std::isfinite(mu) || (mu > 0 && (!(v_slip > 0) || !std::isfinite(v_slip))))
    return fail(ROD_ERR_ARG, "friction needs mu >= 0 and, with mu > 0, a finite slip velocity > 0");
  s->contact.mu = mu;
  s->contact.vslip = mu > 0 ? v_slip : 0.0;
  s->contact.grid_valid = false;  // the contact kernels take the friction law by value
  return ROD_OK;
}

rod_status rod_system_rhs(rod_system* s, double t, double* acc_v, double* acc_w) {
  if (!s || !acc_v || !acc_w) return fail(ROD_ERR_ARG, "null argument");
  if (!s->state_set) return fail(ROD_ERR_STATE, "no state has been set");
  StepParams P = make_params(s);
  if (s->contact.enabled) {
    rod_status st = contact_prepare(s->contact, s->rods_h, s->rods.p, s->x.p, s->N, s->E, s->R, s->stream, s->hook);
    if (st != ROD_OK) return st;
    CUDA_TRY(contact_compute(s->contact, s->x.p, s->v.p, s->rods.p, s->N, s->E, s->R, s->err.p, s->stream, s->hook, false));
    CUDA_TRY(contact_list_invalidate(s->contact, s->stream));  // the cell structures were overwritten
    P.fseg = s->contact.fseg;
  }
  CUDA_TRY(launch_pack_kernel(P, s->shape, MODE_RHS, 1, t, 1.0, 0, acc_v, acc_w, s->stream, s->hook));
  return read_error_word(s);
}

rod_status rod_system_contact_forces(rod_system* s, double* f) {
  if (!s || !f) return fail(ROD_ERR_ARG, "null argument");
  if (!s->state_set) return fail(ROD_ERR_STATE, "no state has been set");
  if (!s->contact.enabled) {
    CUDA_TRY(cudaMemsetAsync(f, 0, 3 * s->N * sizeof(double), s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return ROD_OK;
  }
  rod_status st = contact_prepare(s->contact, s->rods_h, s->rods.p, s->x.p, s->N, s->E, s->R, s->stream, s->hook);
  if (st != ROD_OK) return st;
  CUDA_TRY(contact_compute(s->contact, s->x.p, s->v.p, s->rods.p, s->N, s->E, s->R, s->err.p, s->stream, s->hook, false));
  CUDA_TRY(contact_list_invalidate(s->contact, s->stream));  // the cell structures were overwritten
  CUDA_TRY(contact_node_forces(s->contact, s->rods.p, s->N, s->E, s->R, f, s->stream, s->hook));
  return read_error_word(s);
}

rod_status rod_system_contact_pairs(rod_system* s, int64_t* pairs, int64_t cap, int64_t* n_pairs,
                                    int64_t* n_candidates) {
  if (!s || !n_pairs || cap < 0 || (cap > 0 && !pairs)) return fail(ROD_ERR_ARG, "bad argument");
  if (!s->state_set) return fail(ROD_ERR_STATE, "no state has been set");
  if (!s->contact.enabled) return fail(ROD_ERR_STATE, "contact is disabled");
  rod_status st = contact_prepare(s->contact, s->rods_h, s->rods.p, s->x.p, s->N, s->E, s->R, s->stream, s->hook);
  if (st != ROD_OK) return st;
  // scratch of this debug call only (freed before it returns)
  DevBuf<unsigned long long> counts;
  DevBuf<int64_t> out;
  unsigned long long c[2] = {0, 0};
  cudaError_t e = counts.alloc(2);
  if (!e) e = out.alloc(std::max<int64_t>(2 * cap, 2));
  if (!e)
    e = contact_pairs(s->contact, s->x.p, s->v.p, s->rods.p, s->N, s->E, s->err.p, counts.p, out.p, cap, s->stream,
                      s->hook);
  if (!e) e = contact_list_invalidate(s->contact, s->stream);  // the cell structures were overwritten
  if (!e) e = cudaMemcpyAsync(c, counts.p, sizeof c, cudaMemcpyDeviceToHost, s->stream);
  if (!e) e = cudaStreamSynchronize(s->stream);
  const int64_t n = static_cast<int64_t>(c[0]);
  if (!e && cap > 0 && n > 0)
    e = cudaMemcpy(pairs, out.p, 2 * std::min(n, cap) * sizeof(int64_t), cudaMemcpyDeviceToHost);
  counts.release();
  out.release();
  CUDA_TRY(e);
  st = read_error_word(s);
  if (st != ROD_OK) return st;
  *n_pairs = n;
  if (n_candidates) *n_candidates = static_cast<int64_t>(c[1]);
  return ROD_OK;
}

rod_status rod_system_set_launch(rod_system* s, int32_t elems_per_block, int32_t threads_per_block) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  LaunchShape sh = default_shape(s);
  if (elems_per_block > 0) {
    if (elems_per_block > kMaxCapElems || elems_per_block % 32)
      return fail(ROD_ERR_ARG, "elems_per_block must be a multiple of 32 and <= %d", kMaxCapElems);
    sh.cap_elems = elems_per_block;
    sh.cap_rods = rods_per_pack(s, sh.cap_elems);
  }
  if (threads_per_block > 0) {
    if (threads_per_block > 512 || threads_per_block % 32)
      return fail(ROD_ERR_ARG, "threads_per_block must be a multiple of 32 and <= 512");
    sh.threads = threads_per_block;
  }
  if (step_smem_bytes(sh) > 227 * 1024) return fail(ROD_ERR_ARG, "launch shape needs too much shared memory");
  return build_packs(s, sh);
}

// ---- autotuner: time the step for every valid (elements per block, threads per block) and keep
// the fastest; results are cached per ensemble signature for the process and, when the
// environment variable ROD_AUTOTUNE_CACHE names a file, across processes.
namespace {
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_key(const rod_system* s) {
  int min_n = 1 << 30;
  for (const auto& r : s->rods_h) min_n = std::min(min_n, r.n);
  char buf[160];
  snprintf(buf, sizeof buf, "R%d_E%lld_max%d_min%d_contact%d", s->R, (long long)s->E, s->max_n, min_n,
           s->contact.enabled ? 1 : 0);
  return buf;
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("ROD_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char key[160];
  int cap, thr;
  while (std::fscanf(f, "%159s %d %d", key, &cap, &thr) == 3) g_tune_cache[key] = {cap, thr};
  std::fclose(f);
}

void tune_store() {
  const char* path = std::getenv("ROD_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (const auto& kv : g_tune_cache) std::fprintf(f, "%s %d %d\n", kv.first.c_str(), kv.second.first, kv.second.second);
  std::fclose(f);
}
}  // namespace

rod_status rod_system_autotune(rod_system* s, double dt, int32_t trial_steps, int32_t* best_elems,
                               int32_t* best_threads, double* best_ms) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (!s->state_set) return fail(ROD_ERR_STATE, "no state has been set");
  if (!(dt > 0) || trial_steps < 1) return fail(ROD_ERR_ARG, "need dt > 0 and trial_steps >= 1");
  const std::string key = tune_key(s);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load();
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      rod_status st = rod_system_set_launch(s, it->second.first, it->second.second);
      if (st == ROD_OK) {
        if (best_elems) *best_elems = it->second.first;
        if (best_threads) *best_threads = it->second.second;
        if (best_ms) *best_ms = -1.0;
        return ROD_OK;
      }
    }
  }
  const int64_t ss = state_size(s);
  DevBuf<double> saved;
  CUDA_TRY(saved.alloc(ss));
  CUDA_TRY(pack_state(s, saved.p));
  const double t_saved = s->t;
  const LaunchShape before = s->shape;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int bc = before.cap_elems, bt = before.threads;
  const int caps[] = {192, 224, 256, 288, 320, 384, 448, 512, 640, 768};
  const int thrs[] = {128, 160, 192, 224, 256, 320, 384, 512};
  for (int cap : caps) {
    if (cap < std::min(s->max_n, kMaxCapElems)) continue;
    for (int thr : thrs) {
      if (thr > cap) continue;
      if (rod_system_set_launch(s, cap, thr) != ROD_OK) continue;
      // warm-up step, then the timed trial, then back to the saved state
      if (rod_system_step_async(s, 1, dt) != ROD_OK) continue;
      cudaEventRecord(e0, s->stream);
      if (rod_system_step_async(s, trial_steps, dt) != ROD_OK) continue;
      cudaEventRecord(e1, s->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bc = cap;
        bt = thr;
      }
      CUDA_TRY(unpack_state(s, saved.p));
      s->t = t_saved;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CUDA_TRY(unpack_state(s, saved.p));
  CUDA_TRY(cudaMemsetAsync(s->err.p, 0, sizeof(int), s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->t = t_saved;
  rod_status st = rod_system_set_launch(s, bc, bt);
  if (st != ROD_OK) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = {bc, bt};
    tune_store();
  }
  if (best_elems) *best_elems = bc;
  if (best_threads) *best_threads = bt;
  if (best_ms) *best_ms = best < 1e29f ? best / trial_steps : -1.0;
  return ROD_OK;
}

rod_status rod_system_set_params(rod_system* s, const double* rest_kappa, const double* elem_couple, int on_device) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (rest_kappa) {
    if (s->V == 0) return fail(ROD_ERR_ARG, "the ensemble has no Voronoi points");
    if (!on_device && !finite_all(rest_kappa, 3 * s->V)) return fail(ROD_ERR_ARG, "rest_kappa has non-finite values");
    if (!s->rest_kappa.p) CUDA_TRY(s->rest_kappa.alloc(3 * s->V));
    CUDA_TRY(cudaMemcpyAsync(s->rest_kappa.p, rest_kappa, 3 * s->V * 8, kind, s->stream));
  }
  if (elem_couple) {
    if (!on_device && !finite_all(elem_couple, 3 * s->E)) return fail(ROD_ERR_ARG, "elem_couple has non-finite values");
    if (!s->elem_couple.p) CUDA_TRY(s->elem_couple.alloc(3 * s->E));
    CUDA_TRY(cudaMemcpyAsync(s->elem_couple.p, elem_couple, 3 * s->E * 8, kind, s->stream));
  }
  if (!on_device) CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->ck_valid = false;
  return ROD_OK;
}

rod_status rod_system_forward_checkpointed(rod_system* s, int64_t n_steps, double dt, int32_t every) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (!s->state_set) return fail(ROD_ERR_STATE, "no state has been set");
  if (s->contact.enabled) return fail(ROD_ERR_STATE, "the adjoint does not include contact; disable it first");
  if (n_steps < 1 || every < 1 || !(dt > 0) || !std::isfinite(dt)) return fail(ROD_ERR_ARG, "need n_steps, every >= 1 and dt > 0");
  const int64_t ss = state_size(s);
  const int64_t nck = (n_steps + every - 1) / every;
  if ((int64_t)s->ckpt.n < nck * ss) CUDA_TRY(s->ckpt.alloc(nck * ss));
  StepParams P = make_params(s);
  for (int64_t k = 0; k < n_steps; ++k) {
    if (k % every == 0) CUDA_TRY(pack_state(s, s->ckpt.p + (k / every) * ss));
    CUDA_TRY(launch_pack_kernel(P, s->shape, MODE_STEPS, 1, s->t + k * dt, dt, 1, nullptr, nullptr, s->stream, s->hook));
  }
  s->ck_t0 = s->t;
  s->ck_dt = dt;
  s->ck_steps = n_steps;
  s->ck_every = every;
  s->ck_valid = true;
  s->t += n_steps * dt;
  return read_error_word(s);
}

rod_status rod_system_backward(rod_system* s, const double* gx, const double* gv, const double* gQ, const double* gw,
                               double* grad_kappa0, double* grad_couple) {
  if (!s || !gx || !gv || !gQ || !gw || !grad_kappa0 || !grad_couple) return fail(ROD_ERR_ARG, "null argument");
  if (!s->ck_valid) return fail(ROD_ERR_STATE, "call rod_system_forward_checkpointed first");
  rod_status st = prepare_adjoint_shape(s);
  if (st != ROD_OK) return st;
  if (!s->rest_kappa.p && s->V > 0) {
    CUDA_TRY(s->rest_kappa.alloc(3 * s->V));
    CUDA_TRY(cudaMemsetAsync(s->rest_kappa.p, 0, 3 * s->V * 8, s->stream));
  }
  if (!s->elem_couple.p) {
    CUDA_TRY(s->elem_couple.alloc(3 * s->E));
    CUDA_TRY(cudaMemsetAsync(s->elem_couple.p, 0, 3 * s->E * 8, s->stream));
  }
  const int64_t ss = state_size(s), every = s->ck_every, n = s->ck_steps;
  if ((int64_t)s->seg_states.n < every * ss) CUDA_TRY(s->seg_states.alloc(every * ss));
  if ((int64_t)s->adj.n < ss) CUDA_TRY(s->adj.alloc(ss));
  if ((int64_t)s->final_state.n < ss) CUDA_TRY(s->final_state.alloc(ss));
  CUDA_TRY(pack_state(s, s->final_state.p));
  double* ax = s->adj.p;
  double* av = ax + 3 * s->N;
  double* aQ = ax + 6 * s->N;
  double* aw = aQ + 9 * s->E;
  CUDA_TRY(cudaMemcpyAsync(ax, gx, 3 * s->N * 8, cudaMemcpyDeviceToDevice, s->stream));
  CUDA_TRY(cudaMemcpyAsync(av, gv, 3 * s->N * 8, cudaMemcpyDeviceToDevice, s->stream));
  CUDA_TRY(cudaMemcpyAsync(aQ, gQ, 9 * s->E * 8, cudaMemcpyDeviceToDevice, s->stream));
  CUDA_TRY(cudaMemcpyAsync(aw, gw, 3 * s->E * 8, cudaMemcpyDeviceToDevice, s->stream));
  if (s->V > 0) CUDA_TRY(cudaMemsetAsync(grad_kappa0, 0, 3 * s->V * 8, s->stream));
  CUDA_TRY(cudaMemsetAsync(grad_couple, 0, 3 * s->E * 8, s->stream));
  StepParams P = make_params(s);
  AdjointParams A;
  A.ax = ax;
  A.av = av;
  A.aQ = aQ;
  A.aw = aw;
  A.g_kappa0 = grad_kappa0;
  A.g_couple = grad_couple;
  A.dt = s->ck_dt;
  const int64_t nseg = (n + every - 1) / every;
  for (int64_t seg = nseg - 1; seg >= 0; --seg) {
    const int64_t k0 = seg * every, len = std::min(every, n - k0);
    // recompute the segment's step-start states from its checkpoint
    CUDA_TRY(unpack_state(s, s->ckpt.p + seg * ss));
    for (int64_t k = 0; k < len; ++k) {
      CUDA_TRY(pack_state(s, s->seg_states.p + k * ss));
      if (k + 1 < len)
        CUDA_TRY(launch_pack_kernel(P, s->shape, MODE_STEPS, 1, s->ck_t0 + (k0 + k) * s->ck_dt, s->ck_dt, 1, nullptr,
                                    nullptr, s->stream, s->hook));
    }
    for (int64_t k = len - 1; k >= 0; --k) {
      const double* st0 = s->seg_states.p + k * ss;
      A.P = P;
      A.P.packs = s->adj_packs.p;
      A.P.n_packs = s->adj_n_packs;
      A.P.x = const_cast<double*>(st0);
      A.P.v = const_cast<double*>(st0 + 3 * s->N);
      A.P.Q = const_cast<double*>(st0 + 6 * s->N);
      A.P.w = const_cast<double*>(st0 + 6 * s->N + 9 * s->E);
      A.t = s->ck_t0 + (k0 + k) * s->ck_dt;
      s->hook.before(K_MISC, s->stream);
      cudaError_t e = launch_adjoint_kernel(A, s->adj_shape, s->stream);
      s->hook.after(K_MISC, s->stream);
      CUDA_TRY(e);
    }
  }
  CUDA_TRY(unpack_state(s, s->final_state.p));
  return read_error_word(s);
}

rod_status rod_system_adjoint_of_state(rod_system* s, double* ax, double* av, double* aQ, double* aw) {
  if (!s || !ax || !av || !aQ || !aw) return fail(ROD_ERR_ARG, "null argument");
  if (!s->adj.p) return fail(ROD_ERR_STATE, "no backward pass has run");
  CUDA_TRY(cudaMemcpyAsync(ax, s->adj.p, 3 * s->N * 8, cudaMemcpyDeviceToDevice, s->stream));
  CUDA_TRY(cudaMemcpyAsync(av, s->adj.p + 3 * s->N, 3 * s->N * 8, cudaMemcpyDeviceToDevice, s->stream));
  CUDA_TRY(cudaMemcpyAsync(aQ, s->adj.p + 6 * s->N, 9 * s->E * 8, cudaMemcpyDeviceToDevice, s->stream));
  CUDA_TRY(cudaMemcpyAsync(aw, s->adj.p + 6 * s->N + 9 * s->E, 3 * s->E * 8, cudaMemcpyDeviceToDevice, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return ROD_OK;
}

rod_status rod_system_set_graphs(rod_system* s, int enable) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  s->use_graphs = enable != 0;
  return ROD_OK;
}

rod_status rod_system_profile(rod_system* s, int enable) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  s->prof.reset();
  s->prof.enabled = enable != 0;
  return ROD_OK;
}

int32_t rod_profile_classes(void) { return K_NUM_CLASSES; }

rod_status rod_system_profile_read(rod_system* s, int32_t k, const char** name, double* total_ms, int64_t* launches) {
  if (!s || k < 0 || k >= K_NUM_CLASSES) return fail(ROD_ERR_ARG, "bad system or kernel class");
  s->prof.collect();
  if (name) *name = kernel_class_name(k);
  if (total_ms) *total_ms = s->prof.total_ms[k];
  if (launches) *launches = s->prof.count[k];
  return ROD_OK;
}

rod_status rod_system_launch_count(const rod_system* s, int64_t* launches) {
  if (!s || !launches) return fail(ROD_ERR_ARG, "null argument");
  *launches = s->prof.launches + contact_list_graph_rebuild_launches(s->contact, s->stream);
  return ROD_OK;
}

rod_status rod_system_get_launch(const rod_system* s, int32_t* elems_per_block, int32_t* threads_per_block) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (elems_per_block) *elems_per_block = s->shape.cap_elems;
  if (threads_per_block) *threads_per_block = s->shape.threads;
  return ROD_OK;
}

rod_status rod_system_diagnostics(rod_system* s, double* per_rod, double* totals) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (!s->state_set) return fail(ROD_ERR_STATE, "no state has been set");
  if (!per_rod && !totals) return ROD_OK;
  DiagArgs A;
  A.x = s->x.p;
  A.v = s->v.p;
  A.Q = s->Q.p;
  A.w = s->w.p;
  A.rest_len = s->rest_len.p;
  A.inv_m = s->inv_m.p;
  A.rest_sigma = s->rest_sigma.p;
  A.rest_kappa = s->rest_kappa.p;
  A.rods = s->rods.p;
  A.N = s->N;
  A.E = s->E;
  A.V = s->V;
  A.R = s->R;
  for (int c = 0; c < 3; ++c) A.gravity[c] = s->has_gravity ? s->gravity[c] : 0.0;
  if (!per_rod) {
    if ((int64_t)s->diag_rows.n < 9 * (int64_t)s->R) CUDA_TRY(s->diag_rows.alloc(9 * (size_t)s->R));
    per_rod = s->diag_rows.p;
  }
  A.per_rod = per_rod;
  if (totals && !s->diag_tot.p) CUDA_TRY(s->diag_tot.alloc(6));
  s->hook.before(K_MISC, s->stream);
  CUDA_TRY(launch_diag_rows(A, s->stream));
  s->hook.after(K_MISC, s->stream);
  if (totals) {
    s->hook.before(K_MISC, s->stream);
    CUDA_TRY(launch_diag_totals(per_rod, s->R, s->diag_tot.p, s->stream));
    s->hook.after(K_MISC, s->stream);
    CUDA_TRY(cudaMemcpyAsync(totals, s->diag_tot.p, 6 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
  }
  return ROD_OK;
}

rod_status rod_plan_packs(const int32_t* n_elem, int32_t n_rods, int32_t cap_elems, int32_t cap_rods,
                          int32_t* n_packs, int32_t* n_list, int32_t* n_long, int32_t* packs, int32_t* list) {
  if (!n_elem || n_rods < 1 || cap_elems < 1 || cap_rods < 1) return fail(ROD_ERR_ARG, "need rods and positive capacities");
  std::vector<RodConst> rods(n_rods);
  int64_t e0 = 0;
  for (int r = 0; r < n_rods; ++r) {
    if (n_elem[r] < 1) return fail(ROD_ERR_ARG, "every rod needs at least one element");
    if (e0 + n_elem[r] + r + 1 > INT32_MAX) return fail(ROD_ERR_ARG, "too many elements");
    rods[r] = RodConst{};
    rods[r].n = n_elem[r];
    rods[r].elem0 = static_cast<int32_t>(e0);
    rods[r].node0 = static_cast<int32_t>(e0 + r);
    e0 += n_elem[r];
  }
  const PackPlan plan = plan_packs(rods, cap_elems, cap_rods);
  if (n_packs) *n_packs = static_cast<int32_t>(plan.packs.size());
  if (n_list) *n_list = static_cast<int32_t>(plan.list.size());
  if (n_long) *n_long = static_cast<int32_t>(plan.longs.size());
  if (packs)
    for (size_t k = 0; k < plan.packs.size(); ++k) {
      const Pack& pk = plan.packs[k];
      const int32_t row[10] = {pk.rod0, pk.nrods, pk.elem0, pk.nelem, pk.node0, pk.nnode, pk.vor0, pk.nvor,
                               pk.listed, pk.list_off};
      std::memcpy(packs + 10 * k, row, sizeof row);
    }
  if (list)
    for (size_t k = 0; k < plan.list.size(); ++k) {
      list[2 * k] = plan.list[k].x;
      list[2 * k + 1] = plan.list[k].y;
    }
  return ROD_OK;
}

rod_status rod_system_pack_info(const rod_system* s, int32_t* n_packs, int32_t* n_listed, int32_t* n_long) {
  if (!s) return fail(ROD_ERR_ARG, "null system");
  if (n_packs) *n_packs = s->n_packs;
  if (n_listed) *n_listed = s->n_listed;
  if (n_long) *n_long = static_cast<int32_t>(s->long_packs.size());
  return ROD_OK;
}

}  // extern "C"

namespace rod {
cudaError_t system_clear_error(rod_system* s) { return cudaMemsetAsync(s->err.p, 0, sizeof(int), s->stream); }

rod_status system_view(rod_system* s, SysView* out) {
  if (!s || !out) return fail(ROD_ERR_ARG, "null argument");
  if (!s->state_set) return fail(ROD_ERR_STATE, "no state has been set");
  int min_n = 1 << 30;
  for (const auto& r : s->rods_h) min_n = std::min(min_n, r.n);
  out->x = s->x.p;
  out->v = s->v.p;
  out->Q = s->Q.p;
  out->w = s->w.p;
  out->N = s->N;
  out->E = s->E;
  out->R = s->R;
  out->max_n = s->max_n;
  out->min_n = min_n;
  out->rods = s->rods.p;
  out->rest_len = s->rest_len.p;
  out->contact = s->contact.enabled;
  out->n_packs = s->n_packs;
  out->stream = s->stream;
  out->t = &s->t;
  out->err = s->err.p;
  return ROD_OK;
}
}  // namespace rod

