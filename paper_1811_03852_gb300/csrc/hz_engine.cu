// hz_engine.cu -- host side of the solver: operators, workspaces, the outer
// refinement loop, the inner loop (CUDA-graph while loop or host-driven), and
// the extern "C" entry points declared in include/hz.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "hz_internal.cuh"

using namespace hz;

namespace {

thread_local char g_err[512] = "";

void set_err(cudaError_t e, const char* what, int line) {
  snprintf(g_err, sizeof(g_err), "%s (%d) at hz_engine.cu:%d: %s", cudaGetErrorName(e), (int)e, line, what);
}

#define CK(call)                                                       \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) {                                           \
      set_err(e_, #call, __LINE__);                                    \
      return e_ == cudaErrorMemoryAllocation ? HZ_ERR_OOM : HZ_ERR_CUDA; \
    }                                                                  \
  } while (0)

#define CKS(call)                  \
  do {                             \
    int s_ = (call);               \
    if (s_ != HZ_OK) return s_;    \
  } while (0)

inline int64_t pad64(int64_t n) { return (n + 63) / 64 * 64; }  // 256-byte alignment of FP32 vectors

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct GraphSlot {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct hz_op_s {
  Grid g{};
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  int dev = 0, sms = 0;
  Launch L{};
  double* A7 = nullptr;
  float* ah32 = nullptr;
  float* th32 = nullptr;
  double* ah64 = nullptr;
  double* th64 = nullptr;
  double* invc = nullptr;
  float* w32base = nullptr;
  double* w64base = nullptr;
  Vecs<float> w32{};
  Vecs<double> w64{};
  double* xbuf = nullptr;  // result staging when the caller's x is host memory
  double* xscr = nullptr;  // second buffer of the refinement ping-pong
  double* bbuf = nullptr;  // staging of a host b
  int hb = HB_F32;            // storage of the horizontal bands read by the FP32 BiCGStab kernels
  uint16_t* h16 = nullptr;    // their 16-bit copies [4][pad64(n)] (allocated on first use)
  double* x64buf = nullptr;  // the paper's mixed-precision solver: its FP64 iterate (inner order)
  double* x64nat = nullptr;  // the same scattered to natural order (tri-SOR)
  Ctl* ctl = nullptr;
  Ctl* cfg_h = nullptr;  // pinned: configuration written to ctl
  Ctl* rep_h = nullptr;  // pinned: ctl read back
  Red red{};
  int* err_d = nullptr;
  int* err_h = nullptr;
  int* kerr_d = nullptr;  // bounded-wait error word of kernels launched without a control block
  double* hist_d = nullptr;
  int hist_cap = 0;
  GraphSlot gs[2];  // [0] FP32 inner loop, [1] FP64 inner loop
  // tri-SOR: bands and Thomas factors in colour-compact order ([9][n] per
  // precision, allocated on first use, refreshed after a coefficient update)
  // and the inner-loop graphs, built for one (sweeps, omega) at a time
  float* sor32 = nullptr;
  double* sor64 = nullptr;
  bool sor_ok[2] = {false, false};
  GraphSlot gs_sor[2];
  int gs_sor_sweeps[2] = {0, 0};
  double gs_sor_omega[2] = {0.0, 0.0};
  std::vector<void*> allocs;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // per-kernel profile (CUDA events around every launch; host-driven loop)
  bool prof = false;
  std::vector<cudaEvent_t> pev;
  bool sor_mode = false;  // the current solve uses tri-SOR (compact order)
  long long p_launch[HZ_NUM_KERNELS] = {};
  double p_ms[HZ_NUM_KERNELS] = {};
  double p_bytes[HZ_NUM_KERNELS] = {};
  long long launches = 0;  // kernels launched by the last solve
  FgmWs fgm;               // flexible GMRES workspace (allocated on first use)
  // work vectors of the extra right-hand sides of a batched solve that names
  // this operator more than once (occurrence 1, 2, ...; occurrence 0 uses w32)
  struct RhsWs {
    float* base = nullptr;
    Vecs<float> w{};
    Ctl* ctl = nullptr;
    double* xb = nullptr;
  };
  std::vector<RhsWs> rhs_ws;
  hz_nn nn = nullptr;      // learned stage (not owned)
};

namespace hz {
// l2: the variant uses L2 priorities; cap: its blocks per SM (0: as many as fit)  (hz_launch.cu)
void variant_flags(int prec, int kind, int id, int* l2, int* cap);
}  // namespace hz

namespace {

template <typename T>
T* dalloc(hz_op op, int64_t count, int* st) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, (size_t)count * sizeof(T));
  if (e != cudaSuccess) {
    set_err(e, "cudaMalloc", __LINE__);
    *st = (e == cudaErrorMemoryAllocation) ? HZ_ERR_OOM : HZ_ERR_CUDA;
    return nullptr;
  }
  op->allocs.push_back(p);
  return (T*)p;
}

// h16: the FP32 operator of the BiCGStab T^-1 path, whose stencil kernels read
// the horizontal bands in the operator's band format; the other FP32 paths
// (FGMRES, tri-SOR, batched, training pairs) read the FP32 bands
template <typename T>
Bands<T> bands_of(hz_op op, bool h16 = true);
template <>
Bands<float> bands_of<float>(hz_op op, bool h16) {
  const int64_t n = op->g.n;
  const float* a = op->ah32;
  const float* t = op->th32;
  Bands<float> b{a, a + n, a + 2 * n, a + 3 * n, a + 4 * n, a + 5 * n, t, t + n, t + 2 * n};
  if (h16 && op->hb != HB_F32) {
    b.h16 = op->h16;
    b.h16s = pad64(n);
    b.h16fmt = op->hb;
  }
  return b;
}
template <>
Bands<double> bands_of<double>(hz_op op, bool) {
  const int64_t n = op->g.n;
  const double* a = op->ah64;
  const double* t = op->th64;
  return Bands<double>{a, a + n, a + 2 * n, a + 3 * n, a + 4 * n, a + 5 * n, t, t + n, t + 2 * n};
}

template <typename T>
Vecs<T> carve(T* base, int64_t n) {
  const int64_t s = pad64(n);
  return Vecs<T>{base, base + s, base + 2 * s, base + 3 * s, base + 4 * s,
                 base + 5 * s, base + 6 * s, base + 7 * s, base + 8 * s, base + 9 * s};
}

template <typename T>
Vecs<T>& vecs_of(hz_op op);
template <>
Vecs<float>& vecs_of<float>(hz_op op) { return op->w32; }
template <>
Vecs<double>& vecs_of<double>(hz_op op) { return op->w64; }

int ensure_w64(hz_op op) {
  if (op->w64base) return HZ_OK;
  int st = HZ_OK;
  op->w64base = dalloc<double>(op, 10 * pad64(op->g.n), &st);
  if (!op->w64base) return st;
  op->w64 = carve(op->w64base, op->g.n);
  return HZ_OK;
}

// ---- tri-SOR (colour-compact order) ---------------------------------------
template <typename T>
T*& sor_base(hz_op op);
template <>
float*& sor_base<float>(hz_op op) { return op->sor32; }
template <>
double*& sor_base<double>(hz_op op) { return op->sor64; }

template <typename T>
Bands<T> bands_rb(hz_op op) {
  const int64_t s = pad64(op->g.n);
  const T* b = sor_base<T>(op);
  return Bands<T>{b, b + s, b + 2 * s, b + 3 * s, b + 4 * s, b + 5 * s, b + 6 * s, b + 7 * s, b + 8 * s};
}

// compact copies of the six bands and the three Thomas factors
template <typename T>
int ensure_sor(hz_op op) {
  const int pr = sizeof(T) == 8 ? 1 : 0;
  if (op->sor_ok[pr]) return HZ_OK;
  const int64_t s = pad64(op->g.n);
  T*& base = sor_base<T>(op);
  if (!base) {
    int st = HZ_OK;
    if (!(base = dalloc<T>(op, 9 * s, &st))) return st;
  }
  const Bands<T> a = bands_of<T>(op, false);
  const T* src[9] = {a.E, a.W, a.N, a.S, a.U, a.D, a.m, a.l, a.cp};
  for (int q = 0; q < 9; ++q) CK(launch_rb_copy<T>(op->g, src[q], base + q * s, 1, op->L));
  op->sor_ok[pr] = true;
  return HZ_OK;
}

// One inner BiCGStab iteration with the tri-SOR preconditioner, everything in
// compact order: for each of p and s, the update fused with the first red
// pass, then the remaining 2*sweeps - 1 colour passes ping-ponging between
// the result vector (ph or sh) and t (free at that point); then the full
// matvec with its dots; k_upd is shared with the T^-1 path.
template <typename T>
cudaError_t launch_body_sor(hz_op op, cudaStream_t s, unsigned long long cond, int use_cond, int sweeps,
                            double omega) {
  Launch L = op->L;
  L.stream = s;
  const Bands<T> a = bands_rb<T>(op);
  const Vecs<T>& w = vecs_of<T>(op);
  cudaError_t e;
  for (int half = 0; half < 2; ++half) {
    T* res = half == 0 ? w.ph : w.sh;
    const T* rc = half == 0 ? w.p : w.s;
    // buf[(sw + 1) % 2] receives sweep sw; the last sweep must land in res
    T* buf[2];
    buf[sweeps % 2] = res;
    buf[(sweeps + 1) % 2] = w.t;
    if ((e = launch_sor_first<T>(op->g, a, w, buf[1], omega, half, op->ctl, op->red, L)) != cudaSuccess) return e;
    for (int sw = 0; sw < sweeps; ++sw) {
      T* zin = buf[sw % 2];
      T* zout = buf[(sw + 1) % 2];
      if (sw > 0 &&
          (e = launch_sor_pass<T>(op->g, a, rc, zin, zin, zout, 0, 1, omega, op->ctl, L)) != cudaSuccess)
        return e;
      if ((e = launch_sor_pass<T>(op->g, a, rc, zout, sw > 0 ? zin : nullptr, zout, 1, 1, omega, op->ctl, L)) !=
          cudaSuccess)
        return e;
    }
    if ((e = launch_mv_rb<T>(op->g, a, w, half, op->ctl, op->red, L)) != cudaSuccess) return e;
  }
  return launch_upd<T>(op->g, w, op->ctl, op->red, cond, use_cond, L);
}

// one inner BiCGStab iteration (five launches) on stream s
template <typename T>
cudaError_t launch_body(hz_op op, cudaStream_t s, unsigned long long cond, int use_cond) {
  Launch L = op->L;
  L.stream = s;
  const Bands<T> a = bands_of<T>(op);
  const Vecs<T>& w = vecs_of<T>(op);
  cudaError_t e;
  if ((e = launch_pre_p<T>(op->g, a, w, op->ctl, op->red, L)) != cudaSuccess) return e;
  if ((e = launch_mv_v<T>(op->g, a, w, op->ctl, op->red, L)) != cudaSuccess) return e;
  if ((e = launch_pre_s<T>(op->g, a, w, op->ctl, op->red, L)) != cudaSuccess) return e;
  if ((e = launch_mv_t<T>(op->g, a, w, op->ctl, op->red, L)) != cudaSuccess) return e;
  return launch_upd<T>(op->g, w, op->ctl, op->red, cond, use_cond, L);
}

// Build the inner loop as a graph: one conditional WHILE node whose body is
// one iteration; k_upd sets the condition from the device.
void drop_graph(GraphSlot& gs) {
  if (gs.exec) cudaGraphExecDestroy(gs.exec);
  if (gs.graph) cudaGraphDestroy(gs.graph);
  gs.exec = nullptr;
  gs.graph = nullptr;
}

template <typename F>
int build_loop_graph(hz_op op, GraphSlot& gs, F&& body) {
  if (gs.exec) return HZ_OK;
  CK(cudaGraphCreate(&gs.graph, 0));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, gs.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, gs.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t bg = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(op->cap, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = body((unsigned long long)h);
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(op->cap, &out);
  if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&gs.exec, gs.graph, 0);
  if (e != cudaSuccess || e2 != cudaSuccess) {  // leave the slot empty for the next attempt
    cudaGetLastError();
    drop_graph(gs);
    CK(e != cudaSuccess ? e : e2);
  }
  return HZ_OK;
}

// the tri-SOR loop graph of one precision, rebuilt when (sweeps, omega) change
template <typename T>
int build_graph_sor(hz_op op, int sweeps, double omega) {
  const int pr = sizeof(T) == 8 ? 1 : 0;
  GraphSlot& gs = op->gs_sor[pr];
  if (gs.exec && (op->gs_sor_sweeps[pr] != sweeps || op->gs_sor_omega[pr] != omega)) drop_graph(gs);
  op->gs_sor_sweeps[pr] = sweeps;
  op->gs_sor_omega[pr] = omega;
  return build_loop_graph(op, gs, [&](unsigned long long h) {
    return launch_body_sor<T>(op, op->cap, h, 1, sweeps, omega);
  });
}

template <typename T>
int build_graph(hz_op op) {
  GraphSlot& gs = op->gs[sizeof(T) == 8 ? 1 : 0];
  if (gs.exec) return HZ_OK;
  CK(cudaGraphCreate(&gs.graph, 0));
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, gs.graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, gs.graph, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(op->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = launch_body<T>(op, op->cap, (unsigned long long)h, 1);
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(op->cap, &out);
  if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&gs.exec, gs.graph, 0);
  if (e != cudaSuccess || e2 != cudaSuccess) {  // leave the slot empty for the next attempt
    cudaGetLastError();
    drop_graph(gs);
    CK(e != cudaSuccess ? e : e2);
  }
  return HZ_OK;
}

// Profiled launch: events on the launching stream around the kernel, waited for
// at once, with the launch's algorithmic bytes credited to kernel `kid`.
template <typename F>
int prof_launch(hz_op op, int kid, double bytes, F&& launch) {
  if (op->pev.size() < 2) {
    op->pev.resize(2);
    for (auto& e : op->pev) CK(cudaEventCreate(&e));
  }
  CK(cudaEventRecord(op->pev[0], op->stream));
  CK(launch());
  CK(cudaEventRecord(op->pev[1], op->stream));
  CK(cudaEventSynchronize(op->pev[1]));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, op->pev[0], op->pev[1]));
  op->p_launch[kid] += 1;
  op->p_ms[kid] += ms;
  op->p_bytes[kid] += bytes;
  return HZ_OK;
}

// One inner iteration with every launch timed; the control block is read
// after each launch so that the bytes credited match the work done.
template <typename T>
int profiled_iteration(hz_op op) {
  const double n = (double)op->g.n, B = (double)sizeof(T);
  Launch L = op->L;
  const Bands<T> a = bands_of<T>(op);
  const Vecs<T>& w = vecs_of<T>(op);
  auto state = [&](Ctl* c) -> int {
    CK(cudaMemcpyAsync(c, op->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    return HZ_OK;
  };
  Ctl* c = op->rep_h;
  CKS(state(c));
  if (c->state != ST_RUNNING && c->state != ST_RESTART) return HZ_OK;
  const double bp = c->state == ST_RESTART ? 16 * B : (c->fresh ? 6 * B : 8 * B);
  const bool xz = c->xzero != 0;
  CKS(prof_launch(op, 2, bp * n, [&] { return launch_pre_p<T>(op->g, a, w, op->ctl, op->red, L); }));
  op->launches += 2;  // k_pre_start + k_pre_p
  CKS(state(c));
  if (c->state != ST_RUNNING) return HZ_OK;
  // the stencil kernels read four bands: 2 bytes fewer per band and point when they are 16-bit
  const double hsave = (sizeof(T) == 4 && a.h16fmt != HB_F32) ? 8.0 : 0.0;
  CKS(prof_launch(op, 3, (8 * B - hsave) * n, [&] { return launch_mv_v<T>(op->g, a, w, op->ctl, op->red, L); }));
  CKS(prof_launch(op, 4, 7 * B * n, [&] { return launch_pre_s<T>(op->g, a, w, op->ctl, op->red, L); }));
  // k_mv<1> also takes the half-step test on ||s||: the state after it says
  // which update k_upd makes
  CKS(prof_launch(op, 5, (7 * B - hsave) * n, [&] { return launch_mv_t<T>(op->g, a, w, op->ctl, op->red, L); }));
  op->launches += 3;
  CKS(state(c));
  const bool half = c->state == ST_HALF;
  const double bu = half ? (xz ? 2 : 3) * B : (xz ? 7 : 8) * B;
  CKS(prof_launch(op, 6, bu * n, [&] { return launch_upd<T>(op->g, w, op->ctl, op->red, 0ull, 0, L); }));
  op->launches += 1;
  return HZ_OK;
}

// The tri-SOR iteration with every launch timed (kernel ids 7-9 and 6).
// Algorithmic bytes per point, in units of sizeof(T): k_sor_first 4-6 for the
// p update (13 on a restart) or 3 for s, plus 2 for the red half's Thomas
// factors and z; a colour pass (half the points) 11, 10 without an old
// iterate, 5 without neighbours; k_mv_rb 9.
template <typename T>
int profiled_iteration_sor(hz_op op, int sweeps, double omega) {
  const double n = (double)op->g.n, B = (double)sizeof(T);
  Launch L = op->L;
  const Bands<T> a = bands_rb<T>(op);
  const Vecs<T>& w = vecs_of<T>(op);
  auto state = [&](Ctl* c) -> int {
    CK(cudaMemcpyAsync(c, op->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    return HZ_OK;
  };
  Ctl* c = op->rep_h;
  CKS(state(c));
  if (c->state != ST_RUNNING && c->state != ST_RESTART) return HZ_OK;
  const bool xz = c->xzero != 0;
  for (int half = 0; half < 2; ++half) {
    T* res = half == 0 ? w.ph : w.sh;
    const T* rc = half == 0 ? w.p : w.s;
    T* buf[2];
    buf[sweeps % 2] = res;
    buf[(sweeps + 1) % 2] = w.t;
    double bf = 5.0;
    if (half == 0) bf = c->state == ST_RESTART ? (xz ? 6.0 : 13.0) : (c->fresh ? 4.0 : 6.0);
    CKS(prof_launch(op, 7, bf * B * n, [&] {
      return launch_sor_first<T>(op->g, a, w, buf[1], omega, half, op->ctl, op->red, L);
    }));
    op->launches++;
    CKS(state(c));
    if (c->state != ST_RUNNING) {
      if (half == 0) return HZ_OK;
      break;
    }
    for (int sw = 0; sw < sweeps; ++sw) {
      T* zin = buf[sw % 2];
      T* zout = buf[(sw + 1) % 2];
      if (sw > 0) {
        CKS(prof_launch(op, 8, 5.5 * B * n, [&] {
          return launch_sor_pass<T>(op->g, a, rc, zin, zin, zout, 0, 1, omega, op->ctl, L);
        }));
        op->launches++;
      }
      CKS(prof_launch(op, 8, (sw > 0 ? 5.5 : 5.0) * B * n, [&] {
        return launch_sor_pass<T>(op->g, a, rc, zout, sw > 0 ? zin : nullptr, zout, 1, 1, omega, op->ctl, L);
      }));
      op->launches++;
    }
    CKS(prof_launch(op, 9, 9.0 * B * n, [&] { return launch_mv_rb<T>(op->g, a, w, half, op->ctl, op->red, L); }));
    op->launches++;
    if (half == 0) {
      CKS(state(c));
      if (c->state != ST_RUNNING) break;
    }
  }
  CKS(state(c));
  const bool hs = c->state == ST_HALF;
  const double bu = hs ? (xz ? 2 : 3) * B : (xz ? 7 : 8) * B;
  CKS(prof_launch(op, 6, bu * n, [&] { return launch_upd<T>(op->g, w, op->ctl, op->red, 0ull, 0, L); }));
  op->launches++;
  return HZ_OK;
}

// sweeps > 0: the tri-SOR preconditioner (compact order), else T^-1
template <typename T>
int run_inner(hz_op op, int use_graph, int max_inner, int sweeps = 0, double omega = 0.0) {
  const bool sor = sweeps > 0;
  if (op->prof) {
    for (int it = 0; it < 4 * max_inner + 16; ++it) {
      if (sor)
        CKS(profiled_iteration_sor<T>(op, sweeps, omega));
      else
        CKS(profiled_iteration<T>(op));
      const int st = op->rep_h->state;
      if (st != ST_RUNNING && st != ST_RESTART) break;
    }
    return HZ_OK;
  }
  const int pr = sizeof(T) == 8 ? 1 : 0;
  if (use_graph) {
    if (sor) {
      CKS(build_graph_sor<T>(op, sweeps, omega));
      CK(cudaGraphLaunch(op->gs_sor[pr].exec, op->stream));
    } else {
      CKS(build_graph<T>(op));
      CK(cudaGraphLaunch(op->gs[pr].exec, op->stream));
    }
    return HZ_OK;
  }
  // host-driven: launch iterations in groups and poll the device state
  const int group = 4;
  for (int it = 0; it < 4 * max_inner + 16; it += group) {
    for (int u = 0; u < group; ++u) {
      if (sor)
        CK(launch_body_sor<T>(op, op->stream, 0ull, 0, sweeps, omega));
      else
        CK(launch_body<T>(op, op->stream, 0ull, 0));
    }
    CK(cudaMemcpyAsync(&op->rep_h->state, &op->ctl->state, sizeof(int), cudaMemcpyDeviceToHost, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    const int st = op->rep_h->state;
    if (st != ST_RUNNING && st != ST_RESTART) break;
  }
  return HZ_OK;
}

// ---- flexible GMRES(m) inner solve (FP32 vectors, FP64 scalars) ------------
int ensure_fgm(hz_op op, int m) {
  FgmWs& W = op->fgm;
  if (W.base && W.m >= m) return HZ_OK;
  if (W.base) cudaFree(W.base), W.base = nullptr;
  if (W.vptr) cudaFree(W.vptr), W.vptr = nullptr;
  const int64_t s = pad64(op->g.n);
  CK(cudaMalloc(&W.base, sizeof(float) * (size_t)s * (2 * m + 2)));
  CK(cudaMalloc(&W.vptr, sizeof(float*) * (2 * m + 1)));
  if (!W.part) CK(cudaMalloc(&W.part, sizeof(double) * (size_t)kMaxGrid * (kMaxFgm + 1)));
  if (!W.st) CK(cudaMalloc(&W.st, sizeof(FgmState)));
  std::vector<float*> ptrs(2 * m + 1);
  for (int q = 0; q < 2 * m + 1; ++q) ptrs[q] = W.base + (int64_t)q * s;
  W.w = W.base + (int64_t)(2 * m + 1) * s;
  CK(cudaMemcpy(W.vptr, ptrs.data(), sizeof(float*) * (2 * m + 1), cudaMemcpyHostToDevice));
  W.m = m;
  return HZ_OK;
}

// One inner FGMRES solve of Ahat d = rhs (the right-hand side and its norm come
// from the residual kernel) to relative tolerance eta; d is left in w32.x and
// the control block is updated as the BiCGStab loop would leave it.
// With use_nn the preconditioner is the learned two-stage one,
// z = T^-1 v + sigma NN((v - Ahat T^-1 v) / sigma); it is dropped for plain
// T^-1 (counted in *fallbacks) when the residual estimate has grown above its
// starting value or has not fallen below nn_factor times its value nn_window
// steps earlier.
int run_fgmres(hz_op op, int m, int max_inner, double eta, bool use_nn, int* fallbacks, int nn_window,
               double nn_factor) {
  CKS(ensure_fgm(op, m));
  bool nn_on = use_nn && op->nn != nullptr;
  std::vector<double> rhist;
  FgmWs& W = op->fgm;
  const int64_t n = op->g.n;
  const Launch& L = op->L;
  cudaStream_t s = op->stream;
  const Bands<float> a = bands_of<float>(op, false);
  const Vecs<float>& w32 = op->w32;
  float* const* V = W.vptr;
  float* const* Z = W.vptr + (W.m + 1);
  const int64_t vs = pad64(n);
  auto Vh = [&](int q) { return W.base + (int64_t)q * vs; };
  auto Zh = [&](int q) { return W.base + (int64_t)(W.m + 1 + q) * vs; };
  CK(cudaMemcpyAsync(op->rep_h, op->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double beta0 = std::sqrt(op->rep_h->bnorm2);
  int total = 0, cycles = 0, state = ST_CONVERGED;
  bool xzero = true;
  double resid = beta0;
  if (beta0 > 0.0 && std::isfinite(beta0)) {
    state = ST_MAXIT;
    for (;;) {
      if (cycles == 0) {
        CK(fgm_start(W.st, &op->ctl->bnorm2, s));
        CK(fgm_scale(n, w32.rhs, Vh(0), &op->ctl->bnorm2, 1, L));
      } else {
        CK(fgm_residual(W, op->g, a, w32.rhs, w32.x, Vh(0), &W.st->r2, L));
        CK(fgm_start(W.st, &W.st->r2, s));
        CK(fgm_scale(n, Vh(0), Vh(0), &W.st->r2, 1, L));
      }
      ++cycles;
      int k = 0;
      bool conv = false;
      for (int j = 0; j < W.m && j < m; ++j) {
        CK(launch_tinv<float>(op->g, a, Vh(j), Zh(j), L));        // z_j = M(v_j): T^-1 stage
        if (nn_on) {                                                // learned stage on e1 = v_j - Ahat z1
          CK(fgm_residual(W, op->g, a, Vh(j), Zh(j), W.w, &W.st->r2, L));
          CKS(nn_stage_apply(op->nn, op->g, W.w, &W.st->r2, Zh(j), s));
        }
        CK(launch_matvec_hat<float>(op->g, a, Zh(j), W.w, L));    // w = Ahat z_j
        CK(fgm_multidot(W, n, V, j + 1, W.w, W.st->h1, L));       // CGS, first pass
        CK(fgm_update(W, n, V, j + 1, W.st->h1, W.w, nullptr, L));
        CK(fgm_multidot(W, n, V, j + 1, W.w, W.st->h2, L));       // second pass
        CK(fgm_update(W, n, V, j + 1, W.st->h2, W.w, &W.st->wn2, L));
        CK(fgm_step(W.st, j, s));
        CK(fgm_scale(n, W.w, Vh(j + 1), &W.st->wn2, 1, L));       // v_(j+1) = w / ||w||
        ++total;
        k = j + 1;
        CK(cudaMemcpyAsync(&op->rep_h->snorm2, &W.st->resid, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        resid = op->rep_h->snorm2;
        if (!std::isfinite(resid)) {
          state = ST_NONFINITE;
          break;
        }
        if (resid <= eta * beta0) {
          conv = true;
          break;
        }
        rhist.push_back(resid);
        if (nn_on) {
          const size_t h = rhist.size();
          const size_t wnd = (size_t)nn_window;
          if (resid > beta0 || (h > wnd && resid > nn_factor * rhist[h - wnd - 1])) {
            nn_on = false;  // the learned stage is not helping: plain T^-1 from here on
            if (fallbacks) ++*fallbacks;
          }
        }
        if (total >= max_inner) break;
      }
      if (state == ST_NONFINITE) break;
      CK(fgm_solve_update(W.st, n, Z, k, w32.x, xzero ? 1 : 0, L));
      xzero = false;
      if (conv) {
        state = ST_CONVERGED;
        break;
      }
      if (total >= max_inner) break;
    }
  }
  // leave the control block as the BiCGStab loop would
  CK(cudaMemcpyAsync(op->rep_h, op->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  Ctl c = *op->rep_h;
  c.iter = total;
  c.restarts = cycles > 0 ? cycles - 1 : 0;
  c.state = state;
  c.xzero = xzero ? 1 : 0;
  c.rnorm2 = resid * resid;
  *op->cfg_h = c;
  CK(cudaMemcpyAsync(op->ctl, op->cfg_h, sizeof(Ctl), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  return HZ_OK;
}

int do_setup(hz_op op, const double* coeffs) {
  const int64_t n = op->g.n;
  const bool dev = is_device_ptr(coeffs);
  CK(cudaMemcpyAsync(op->A7, coeffs, sizeof(double) * 7 * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     op->stream));
  CK(cudaMemsetAsync(op->err_d, 0, sizeof(int), op->stream));
  op->sor_ok[0] = op->sor_ok[1] = false;  // compact copies are redone on next use
  SetupOut o{op->ah32, op->th32, op->ah64, op->th64, op->invc, op->err_d};
  if (op->prof)
    CKS(prof_launch(op, 0, 164.0 * (double)n, [&] { return launch_setup(op->g, op->A7, o, op->L); }));
  else
    CK(launch_setup(op->g, op->A7, o, op->L));
  if (op->hb != HB_F32) CK(launch_h16(op->g, op->ah64, op->h16, pad64(n), op->hb, op->L));
  CK(cudaMemcpyAsync(op->err_h, op->err_d, sizeof(int), cudaMemcpyDeviceToHost, op->stream));
  CK(cudaStreamSynchronize(op->stream));
  if (*op->err_h) {
    snprintf(g_err, sizeof(g_err), "operator rejected (flags %d: 1 zero/non-finite coefficient, 2 flux across a "
             "pole or the top/bottom, 4 tridiagonal factor breakdown)", *op->err_h);
    return HZ_ERR_INVALID;
  }
  return HZ_OK;
}

void free_op(hz_op op) {
  if (!op) return;
  for (auto& gs : op->gs_sor) drop_graph(gs);
  for (auto& gs : op->gs) {
    if (gs.exec) cudaGraphExecDestroy(gs.exec);
    if (gs.graph) cudaGraphDestroy(gs.graph);
  }
  for (void* p : op->allocs) cudaFree(p);
  if (op->fgm.base) cudaFree(op->fgm.base);
  if (op->fgm.vptr) cudaFree(op->fgm.vptr);
  if (op->fgm.part) cudaFree(op->fgm.part);
  if (op->fgm.st) cudaFree(op->fgm.st);
  for (auto& r : op->rhs_ws) {
    if (r.base) cudaFree(r.base);
    if (r.ctl) cudaFree(r.ctl);
    if (r.xb) cudaFree(r.xb);
  }
  if (op->cfg_h) cudaFreeHost(op->cfg_h);
  if (op->rep_h) cudaFreeHost(op->rep_h);
  if (op->err_h) cudaFreeHost(op->err_h);
  if (op->cap) cudaStreamDestroy(op->cap);
  if (op->ev0) cudaEventDestroy(op->ev0);
  if (op->ev1) cudaEventDestroy(op->ev1);
  delete op;
}

// ---- column-kernel variants -------------------------------------------------
bool variant_ok(int prec, int kind, int id, const Grid& g) {
  int v = 1, u = 1;
  variant_shape(prec, kind, id, &v, &u);
  if (kind == 0 && variant_park_mode(prec, id) == kParkBulk) return prec == 0 && thomas_bulk_ok(g);
  if (variant_parks_smem(prec, kind, id) && (size_t)g.nz * kBS * v * (prec ? 8 : 4) > 200 * 1024) return false;
  return g.nx % v == 0;
}

// The launch shape used until the autotuner picks one (and kept by it unless
// another is clearly faster), the best measured on GB300 inside the N1280
// iteration: for the Thomas kernels, the variant that parks its forward sweep
// under L2 priorities with two columns per thread and no block cap; for the
// stencil kernels, the L2-priority variant with two columns per thread and the
// deepest batch.  Rows whose length two does not divide: the widest vector
// the row length allows.
int default_variant(int prec, int kind, int nx) {
  int best = 0, bestv = 0;
  if (nx % 2 == 0) {
    int pick = -1, pu = 0;
    for (int i = 0; i < num_variants(prec, kind); ++i) {
      int v = 1, u = 1, l2 = 0, cap = 0;
      variant_shape(prec, kind, i, &v, &u);
      variant_flags(prec, kind, i, &l2, &cap);
      if (v == 2 && l2 && cap == 0 && u > pu) {
        pick = i;
        pu = u;
      }
    }
    if (pick >= 0) return pick;
  }
  for (int i = 0; i < num_variants(prec, kind); ++i) {
    int v = 1, u = 1;
    variant_shape(prec, kind, i, &v, &u);
    if (nx % v == 0 && v > bestv && !variant_parks_smem(prec, kind, i) &&
        !(kind == 0 && variant_park_mode(prec, i) == kParkBulk)) {
      best = i;
      bestv = v;
    }
  }
  return best;
}

void device_name(char* out, size_t cap) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp pr;
  if (cudaGetDeviceProperties(&pr, dev) == cudaSuccess) {
    snprintf(out, cap, "%s", pr.name);
    for (char* c = out; *c; ++c)
      if (*c == ' ' || *c == '|') *c = '_';
  } else {
    snprintf(out, cap, "unknown");
  }
}

// Autotuner cache: a text file (path in HZ_AUTOTUNE_CACHE), one line per
// (device, grid, precision, kernel kind): "device|nx|ny|nz|prec|kind variant".
std::mutex g_tune_mu;

void tune_key(hz_op op, int prec, int kind, char* key, size_t cap) {
  char dn[128];
  device_name(dn, sizeof(dn));
  snprintf(key, cap, "%s|%d|%d|%d|%d|%d", dn, op->g.nx, op->g.ny, op->g.nz, prec, kind);
}

void load_tuned(hz_op op) {
  const char* path = getenv("HZ_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    char key[400];
    int var = -1;
    if (sscanf(line, "%399s %d", key, &var) != 2) continue;
    for (int pr = 0; pr < 2; ++pr)
      for (int kind = 0; kind < 5; ++kind) {
        char want[400];
        tune_key(op, pr, kind, want, sizeof(want));
        if (strcmp(want, key) != 0 || var < 0) continue;
        if (kind < 2 && var < num_variants(pr, kind) && variant_ok(pr, kind, var, op->g))
          (kind == 0 ? op->L.vpre : op->L.vmv)[pr] = var;
        else if (kind >= 2 && sor_variant_ok(pr, kind - 2, var, op->g.nx))
          op->L.vsor[pr][kind - 2] = var;
      }
  }
  fclose(f);
}

void store_tuned(hz_op op) {
  const char* path = getenv("HZ_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE* f = fopen(path, "a");
  if (!f) return;
  for (int pr = 0; pr < 2; ++pr)
    for (int kind = 0; kind < 5; ++kind) {
      char key[400];
      tune_key(op, pr, kind, key, sizeof(key));
      fprintf(f, "%s %d\n", key, kind < 2 ? (kind == 0 ? op->L.vpre : op->L.vmv)[pr] : op->L.vsor[pr][kind - 2]);
    }
  fclose(f);
}

// test hooks of the batched solve (bounded grid-barrier wait)
long long g_batch_timeout_ns = 2000000000LL;
int g_batch_leave_block = -1;
int g_batch_vec = 0;  // columns per thread of the persistent kernel (0: chosen per batch)

// global scratch for hz_dot (per device)
std::mutex g_dot_mu;
struct DotScratch {
  double* partials = nullptr;
  unsigned* ticket = nullptr;
  double* out = nullptr;
  double* out_h = nullptr;
};
DotScratch g_dot[64];

}  // namespace

// ===========================================================================
extern "C" {

int hz_version(void) { return HZ_ABI_VERSION; }

const char* hz_last_error(void) { return g_err; }

const char* hz_status_str(int s) {
  switch (s) {
    case HZ_OK: return "ok";
    case HZ_ERR_INVALID: return "invalid argument or operator";
    case HZ_ERR_CUDA: return "CUDA error";
    case HZ_ERR_OOM: return "out of device memory";
    case HZ_ERR_NOT_CONVERGED: return "not converged";
    case HZ_ERR_BREAKDOWN: return "Krylov breakdown";
    case HZ_ERR_NONFINITE: return "non-finite value";
    case HZ_ERR_TIMEOUT: return "device wait timed out";
    case HZ_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

void hz_default_params(hz_solve_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->tol = 1e-8;
  p->inner_tol = 0.0;  // 0 = mode default
  p->mode = HZ_MODE_MIXED_IR;
  p->precond = HZ_PRE_TRI;
  p->krylov = HZ_KRYLOV_BICGSTAB;
  p->max_outer = 10;
  p->max_inner = 1000;
  p->restart = 150;
  p->fgmres_m = 30;
  p->use_graph = 1;
  p->record_history = 0;
  p->sor_sweeps = 3;
  p->sor_omega = 1.5;
  p->dot_fp32 = 0;
  p->nn_window = 10;
  p->nn_factor = 0.5;
}

int hz_op_create(int nx, int ny, int nz, const double* coeffs, void* stream, hz_op* out) {
  if (!out) return HZ_ERR_INVALID;
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || nz > HZ_MAX_LEVELS || !coeffs) return HZ_ERR_INVALID;
  const int64_t n = (int64_t)nx * ny * nz;
  if (n > ((int64_t)1 << 40)) return HZ_ERR_INVALID;
  hz_op op = new hz_op_s();
  op->g = Grid{nx, ny, nz, (int64_t)nx * ny, n};
  op->stream = (cudaStream_t)stream;
  int st = HZ_OK;
  auto fail = [&](int s) {
    free_op(op);
    return s;
  };
  if (cudaGetDevice(&op->dev) != cudaSuccess) return fail(HZ_ERR_CUDA);
  cudaDeviceGetAttribute(&op->sms, cudaDevAttrMultiProcessorCount, op->dev);
  if (cudaStreamCreateWithFlags(&op->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(HZ_ERR_CUDA);
  cudaEventCreate(&op->ev0);
  cudaEventCreate(&op->ev1);
  // launch shapes: each kernel fills the SMs to its own occupancy (grid-stride loops)
  op->L = Launch{op->sms, (op->g.ncol + kBS - 1) / kBS, (n / 4 + 255) / 256 + 1, op->stream};
  op->L.nz = nz;
  warm_launch_cache(op->L);
  for (int pr = 0; pr < 2; ++pr) {
    op->L.vpre[pr] = default_variant(pr, 0, nx);
    op->L.vmv[pr] = default_variant(pr, 1, nx);
  }
  load_tuned(op);
  if (!(op->A7 = dalloc<double>(op, 7 * n, &st))) return fail(st);
  if (!(op->ah32 = dalloc<float>(op, 6 * n, &st))) return fail(st);
  if (!(op->th32 = dalloc<float>(op, 3 * n, &st))) return fail(st);
  if (!(op->ah64 = dalloc<double>(op, 6 * n, &st))) return fail(st);
  if (!(op->th64 = dalloc<double>(op, 3 * n, &st))) return fail(st);
  if (!(op->invc = dalloc<double>(op, n, &st))) return fail(st);
  if (!(op->w32base = dalloc<float>(op, 10 * pad64(n), &st))) return fail(st);
  op->w32 = carve(op->w32base, n);
  if (!(op->xscr = dalloc<double>(op, n, &st))) return fail(st);
  if (!(op->ctl = dalloc<Ctl>(op, 1, &st))) return fail(st);
  if (!(op->red.partials = dalloc<double>(op, (int64_t)kMaxGrid * kMaxND, &st))) return fail(st);
  if (!(op->red.ticket = dalloc<unsigned>(op, 1, &st))) return fail(st);
  if (!(op->err_d = dalloc<int>(op, 1, &st))) return fail(st);
  if (!(op->kerr_d = dalloc<int>(op, 1, &st))) return fail(st);
  if (cudaMemsetAsync(op->kerr_d, 0, sizeof(int), op->stream) != cudaSuccess) return fail(HZ_ERR_CUDA);
  op->L.err = op->kerr_d;
  if (cudaMallocHost(&op->cfg_h, sizeof(Ctl)) != cudaSuccess) return fail(HZ_ERR_OOM);
  if (cudaMallocHost(&op->rep_h, sizeof(Ctl)) != cudaSuccess) return fail(HZ_ERR_OOM);
  if (cudaMallocHost(&op->err_h, sizeof(int)) != cudaSuccess) return fail(HZ_ERR_OOM);
  if (cudaMemsetAsync(op->red.ticket, 0, sizeof(unsigned), op->stream) != cudaSuccess) return fail(HZ_ERR_CUDA);
  if (cudaMemsetAsync(op->ctl, 0, sizeof(Ctl), op->stream) != cudaSuccess) return fail(HZ_ERR_CUDA);
  st = do_setup(op, coeffs);
  if (st != HZ_OK) return fail(st);
  *out = op;
  return HZ_OK;
}

int hz_op_update(hz_op op, const double* coeffs) {
  if (!op || !coeffs) return HZ_ERR_INVALID;
  return do_setup(op, coeffs);
}

int hz_op_destroy(hz_op op) {
  if (!op) return HZ_OK;
  cudaStreamSynchronize(op->stream);
  free_op(op);
  return HZ_OK;
}

int hz_op_set_band_format(hz_op op, int fmt) {
  if (!op || (fmt != HZ_BANDS_FP32 && fmt != HZ_BANDS_BF16 && fmt != HZ_BANDS_FP16)) return HZ_ERR_INVALID;
  const int hb = fmt == HZ_BANDS_BF16 ? HB_BF16 : fmt == HZ_BANDS_FP16 ? HB_FP16 : HB_F32;
  if (hb == op->hb) return HZ_OK;
  if (hb != HB_F32) {
    int st = HZ_OK;
    if (!op->h16 && !(op->h16 = dalloc<uint16_t>(op, 4 * pad64(op->g.n), &st))) return st;
    CK(launch_h16(op->g, op->ah64, op->h16, pad64(op->g.n), hb, op->L));
    CK(cudaStreamSynchronize(op->stream));
  }
  op->hb = hb;
  drop_graph(op->gs[0]);  // the captured FP32 loop launches the previous format's kernels
  return HZ_OK;
}

int hz_op_get_band_format(hz_op op, int* fmt) {
  if (!op || !fmt) return HZ_ERR_INVALID;
  *fmt = op->hb == HB_BF16 ? HZ_BANDS_BF16 : op->hb == HB_FP16 ? HZ_BANDS_FP16 : HZ_BANDS_FP32;
  return HZ_OK;
}

int hz_op_set_nn(hz_op op, hz_nn nn) {
  if (!op) return HZ_ERR_INVALID;
  op->nn = nn;
  return HZ_OK;
}

int hz_nn_make_pair(hz_op op, const double* b, const double* xk, const double* x_star, float* in, float* target,
                    double* sigma) {
  if (!op || !b || !xk || !x_star || !in || !target) return HZ_ERR_INVALID;
  CKS(ensure_fgm(op, 1));
  const int64_t n = op->g.n;
  cudaStream_t s = op->stream;
  FgmWs& W = op->fgm;
  Vecs<float>& w = op->w32;
  // r = b - A x_k (FP64) into the refinement scratch
  CK(launch_residual<float>(op->g, op->A7, op->invc, b, xk, nullptr, nullptr, w.rhs, op->xscr, 0, op->ctl, op->red,
                            op->L));
  CK(nn_pair_launch(n, op->A7, b, xk, x_star, op->xscr, w.r, w.s, nullptr, nullptr, nullptr, nullptr, nullptr, 0, s));
  CK(launch_tinv<float>(op->g, bands_of<float>(op, false), w.r, w.p, op->L));                   // z1 = T^-1 r
  CK(fgm_residual(W, op->g, bands_of<float>(op, false), w.r, w.p, w.v, &W.st->r2, op->L));     // e1 = r - Ahat z1
  CK(nn_pair_launch(n, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, w.s, w.v, w.p, &W.st->r2, in, target, 1,
                    s));
  CK(cudaMemcpyAsync(&op->rep_h->snorm2, &W.st->r2, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (sigma) *sigma = std::sqrt(op->rep_h->snorm2 / (double)n);
  return HZ_OK;
}

int hz_op_dims(hz_op op, int* nx, int* ny, int* nz) {
  if (!op) return HZ_ERR_INVALID;
  if (nx) *nx = op->g.nx;
  if (ny) *ny = op->g.ny;
  if (nz) *nz = op->g.nz;
  return HZ_OK;
}

int hz_solve(hz_op op, const double* b, const double* x0, double* x, const hz_solve_params* pp,
             hz_solve_info* info) {
  if (!op || !b || !x) return HZ_ERR_INVALID;
  hz_solve_params p;
  if (pp)
    p = *pp;
  else
    hz_default_params(&p);
  if (!(p.tol > 0.0) || p.max_outer < 0 || p.max_inner < 1 || p.restart < 1) return HZ_ERR_INVALID;
  if (p.mode != HZ_MODE_FP64 && p.mode != HZ_MODE_MIXED_IR && p.mode != HZ_MODE_PAPER_MP &&
      p.mode != HZ_MODE_PAPER_DP)
    return HZ_ERR_INVALID;
  // the two solvers of the paper's Sec. 4 comparison: one BiCGStab solve each,
  // halting on its own test, no refinement; the mixed one keeps x in FP64
  const bool paper = (p.mode == HZ_MODE_PAPER_MP || p.mode == HZ_MODE_PAPER_DP);
  const bool mp64 = (p.mode == HZ_MODE_PAPER_MP);
  if (paper && (p.krylov != HZ_KRYLOV_BICGSTAB || p.precond == HZ_PRE_TRI_NN)) return HZ_ERR_UNSUPPORTED;
  if (p.dot_fp32 && (p.mode == HZ_MODE_FP64 || p.mode == HZ_MODE_PAPER_DP)) return HZ_ERR_UNSUPPORTED;
  if (p.krylov != HZ_KRYLOV_BICGSTAB && p.krylov != HZ_KRYLOV_FGMRES) return HZ_ERR_INVALID;
  if (p.krylov == HZ_KRYLOV_FGMRES && (p.mode != HZ_MODE_MIXED_IR || p.fgmres_m < 1 || p.fgmres_m > kMaxFgm))
    return HZ_ERR_UNSUPPORTED;
  if (p.precond != HZ_PRE_TRI && p.precond != HZ_PRE_TRI_NN && p.precond != HZ_PRE_TRISOR) return HZ_ERR_INVALID;
  // the learned stage is not a fixed linear operator: it needs the flexible solver and a network
  if (p.precond == HZ_PRE_TRI_NN && (p.krylov != HZ_KRYLOV_FGMRES || !op->nn)) return HZ_ERR_UNSUPPORTED;
  if (p.precond == HZ_PRE_TRI_NN && (p.nn_window < 0 || !(p.nn_factor > 0.0 && p.nn_factor <= 1.0)))
    return HZ_ERR_INVALID;
  const bool sor = (p.precond == HZ_PRE_TRISOR);
  if (sor) {
    if (p.sor_sweeps < 1 || p.sor_sweeps > 64 || !(p.sor_omega > 0.0 && p.sor_omega < 2.0)) return HZ_ERR_INVALID;
    if (p.krylov != HZ_KRYLOV_BICGSTAB || op->g.nx % 2 != 0) return HZ_ERR_UNSUPPORTED;
  }
  const bool fp32_mode = (p.mode == HZ_MODE_MIXED_IR || p.mode == HZ_MODE_PAPER_MP);
  // precision of the inner solves: FP32 in mixed mode until a refinement step
  // stalls (then FP64 for the rest of the solve, see below)
  bool fp32 = fp32_mode;
  // FP64 mode is plain BiCGStab to tol (one inner solve; the outer check adds a
  // step only if the scaled residual and the true one disagree)
  // (the paper's mixed-precision solver halts its one solve at tol, Sec. 3)
  const double eta = p.inner_tol > 0.0 ? p.inner_tol : ((fp32 && !paper) ? 1e-4 : p.tol);
  const int64_t n = op->g.n;
  const size_t bytes = sizeof(double) * (size_t)n;
  cudaStream_t s = op->stream;
  if (!fp32) CKS(ensure_w64(op));
  if (sor) CKS(fp32 ? ensure_sor<float>(op) : ensure_sor<double>(op));
  if (p.record_history) {
    const int cap = std::max(1, p.max_inner * std::max(1, p.max_outer));
    if (cap > op->hist_cap) {
      int st = HZ_OK;
      op->hist_d = dalloc<double>(op, cap, &st);
      if (!op->hist_d) return st;
      op->hist_cap = cap;
    }
  }
  // pointer kinds
  const bool b_dev = is_device_ptr(b);
  const bool x_dev = is_device_ptr(x);
  const bool x0_dev = x0 && is_device_ptr(x0);
  int st = HZ_OK;
  const double* bd = b;
  if (!b_dev) {
    if (!op->bbuf && !(op->bbuf = dalloc<double>(op, n, &st))) return st;
    CK(cudaMemcpyAsync(op->bbuf, b, bytes, cudaMemcpyHostToDevice, s));
    bd = op->bbuf;
  }
  double* XA = x;
  if (!x_dev) {
    if (!op->xbuf && !(op->xbuf = dalloc<double>(op, n, &st))) return st;
    XA = op->xbuf;
  }
  double* XB = op->xscr;
  if (mp64) {
    if (!op->x64buf && !(op->x64buf = dalloc<double>(op, n, &st))) return st;
    if (sor && !op->x64nat && !(op->x64nat = dalloc<double>(op, n, &st))) return st;
  }
  CK(cudaEventRecord(op->ev0, s));
  const double* cur = nullptr;
  if (x0) {
    if (x0_dev) {
      cur = x0;
    } else {
      CK(cudaMemcpyAsync(XA, x0, bytes, cudaMemcpyHostToDevice, s));
      cur = XA;
    }
  }
  // configuration of the control block
  Ctl* cfg = op->cfg_h;
  memset(cfg, 0, sizeof(Ctl));
  cfg->eta = eta;
  cfg->maxit = p.max_inner;
  cfg->body_limit = 4 * p.max_inner + 64;
  cfg->restart_every = p.restart;
  cfg->hist = p.record_history ? op->hist_d : nullptr;
  cfg->hist_cap = p.record_history ? op->hist_cap : 0;
  cfg->xzero = 1;
  cfg->state = ST_CONVERGED;
  cfg->x64 = mp64 ? op->x64buf : nullptr;
  cfg->dot32 = p.dot_fp32 ? 1 : 0;
  CK(cudaMemcpyAsync(op->ctl, cfg, sizeof(Ctl), cudaMemcpyHostToDevice, s));

  // tri-SOR: the inner vectors are in colour-compact order; the inner solution
  // is scattered to natural order (into s) before the residual and the new
  // inner right-hand side (written to t) gathered back into rhs after it
  auto residual = [&](const double* xin, double* xout, bool with_delta) -> int {
    const double ds = fp32 ? 4.0 : 8.0;
    const double dd = mp64 ? 8.0 : ds;  // bytes of a correction value
    auto step = [&](int kid, double bytes, auto&& launch) -> int {
      if (op->prof)
        CKS(prof_launch(op, kid, bytes * (double)n, launch));
      else
        CK(launch());
      op->launches++;
      return HZ_OK;
    };
    auto rb = [&](int to_compact) -> cudaError_t {
      if (mp64 && !to_compact) return launch_rb_copy<double>(op->g, op->x64buf, op->x64nat, 0, op->L);
      if (fp32)
        return to_compact ? launch_rb_copy<float>(op->g, op->w32.t, op->w32.rhs, 1, op->L)
                          : launch_rb_copy<float>(op->g, op->w32.x, op->w32.s, 0, op->L);
      return to_compact ? launch_rb_copy<double>(op->g, op->w64.t, op->w64.rhs, 1, op->L)
                        : launch_rb_copy<double>(op->g, op->w64.x, op->w64.s, 0, op->L);
    };
    if (sor && with_delta) CKS(step(10, 2 * dd, [&] { return rb(0); }));
    auto go = [&]() -> cudaError_t {
      if (mp64 && with_delta)
        return launch_residual_x64(op->g, op->A7, op->invc, bd, xin, xout, sor ? op->x64nat : op->x64buf,
                                   sor ? op->w32.t : op->w32.rhs, op->ctl, op->red, op->L);
      if (fp32) {
        const Vecs<float>& w = op->w32;
        return launch_residual<float>(op->g, op->A7, op->invc, bd, xin, xout,
                                      with_delta ? (sor ? w.s : w.x) : nullptr, sor ? w.t : w.rhs, nullptr, 0,
                                      op->ctl, op->red, op->L);
      }
      const Vecs<double>& w = op->w64;
      return launch_residual<double>(op->g, op->A7, op->invc, bd, xin, xout, with_delta ? (sor ? w.s : w.x) : nullptr,
                                     sor ? w.t : w.rhs, nullptr, 0, op->ctl, op->red, op->L);
    };
    // algorithmic bytes: C band, b, rhs; plus the other six bands, x, d and x out for a stencil pass
    double bp = 8 + 8 + ds;
    if (xin || with_delta) bp += 48 + (xin ? 8 : 0) + (with_delta ? dd : 0) + (xout ? 8 : 0);
    CKS(step(1, bp, go));
    if (sor) CKS(step(10, 2 * ds, [&] { return rb(1); }));
    CK(cudaMemcpyAsync(op->rep_h, op->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return HZ_OK;
  };

  op->launches = 0;
  CKS(residual(cur, nullptr, false));
  const double bb = op->rep_h->res_bb;
  double R = bb > 0.0 ? std::sqrt(op->rep_h->res_rr / bb) : std::sqrt(op->rep_h->res_rr);
  int outer = 0, inner_total = 0, restarts = 0, status = HZ_OK, fallbacks = 0, retries = 0;
  double scaled = 0.0, Rprev = R;
  int stall = 0;
  // One retry in FP64 (mixed BiCGStab only): when an FP32 refinement step fails
  // to halve R, or its inner solve met a non-finite value while the FP64
  // residual is finite (the 32-bit range was exceeded), the remaining inner
  // solves run in FP64 from the current x; a later stall ends the solve.
  auto retry_fp64 = [&]() -> int {
    fp32 = false;
    ++retries;
    stall = 1;
    CKS(ensure_w64(op));
    if (sor) CKS(ensure_sor<double>(op));
    CKS(residual(cur, nullptr, false));  // r = b - A x again, FP64 right-hand side for the inner solve
    return HZ_OK;
  };
  const bool can_retry = fp32_mode && !paper && p.krylov == HZ_KRYLOV_BICGSTAB;
  // no refinement in the paper's solver: one inner solve, then the report
  const int max_outer = paper ? std::min(p.max_outer, 1) : p.max_outer;
  for (;;) {
    if (!std::isfinite(R)) { status = HZ_ERR_NONFINITE; break; }
    if (R <= p.tol) { status = HZ_OK; break; }
    if (outer >= max_outer) { status = HZ_ERR_NOT_CONVERGED; break; }
    if (p.krylov == HZ_KRYLOV_FGMRES)
    {
      CKS(run_fgmres(op, p.fgmres_m, p.max_inner, eta, p.precond == HZ_PRE_TRI_NN, &fallbacks,
                     p.nn_window > 0 ? p.nn_window : p.fgmres_m, p.nn_factor));
      if (p.precond == HZ_PRE_TRI_NN) CKS(nn_stage_status(op->nn, op->stream));
    }
    else if (fp32)
      CKS(run_inner<float>(op, p.use_graph, p.max_inner, sor ? p.sor_sweeps : 0, p.sor_omega));
    else
      CKS(run_inner<double>(op, p.use_graph, p.max_inner, sor ? p.sor_sweeps : 0, p.sor_omega));
    double* next = (cur == XA) ? XB : XA;
    CKS(residual(cur, next, true));
    const Ctl& rp = *op->rep_h;
    if (rp.kerr) {
      snprintf(g_err, sizeof(g_err), "inner solve: a bounded wait of a bulk-copy kernel ran out");
      status = HZ_ERR_TIMEOUT;
      break;
    }
    // launches per inner iteration: 6 with T^-1; with tri-SOR 2 first-pass
    // kernels, 2 (2 sweeps - 1) colour passes, 2 matvecs and k_upd
    const long long per_it = sor ? 4LL * p.sor_sweeps + 3 : 6LL;
    if (!op->prof) op->launches += per_it * std::max(1, rp.last_iter);
    inner_total += rp.last_iter;
    restarts += rp.last_restarts;
    scaled = rp.last_bnorm2 > 0.0 ? std::sqrt(rp.last_rnorm2 / rp.last_bnorm2) : 0.0;
    cur = next;
    ++outer;
    const double Rn = bb > 0.0 ? std::sqrt(rp.res_rr / bb) : std::sqrt(rp.res_rr);
    if (rp.last_state == ST_NONFINITE) {
      R = Rn;
      // the FP32 inner solve overflowed although the FP64 residual is finite
      // (the residual pass then leaves x unchanged): retry in FP64
      if (can_retry && fp32 && retries == 0 && std::isfinite(R) && outer < max_outer) {
        CKS(retry_fp64());
        continue;
      }
      status = HZ_ERR_NONFINITE;
      break;
    }
    R = Rn;
    if (paper) {
      // the paper's solver ends after its one solve; its own halting test (the
      // recursive residual of the scaled system, Sec. 3) decides the status,
      // and R above is reported as computed
      status = rp.last_state == ST_CONVERGED ? HZ_OK : HZ_ERR_NOT_CONVERGED;
      break;
    }
    // stagnation: a refinement step that does not halve R; two in a row end the
    // solve, and in mixed mode the first one is retried in FP64
    if (R > 0.5 * Rprev && R > p.tol) {
      if (can_retry && fp32 && retries == 0 && outer < max_outer) {
        CKS(retry_fp64());
      } else if (++stall >= 2) {
        status = HZ_ERR_NOT_CONVERGED;
        break;
      }
    } else {
      stall = 0;
    }
    Rprev = R;
  }
  // deliver x
  if (cur == nullptr) {
    if (x_dev)
      CK(cudaMemsetAsync(x, 0, bytes, s));
    else
      memset(x, 0, bytes);
  } else if (x_dev) {
    if (cur != x) CK(cudaMemcpyAsync(x, cur, bytes, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(cudaMemcpyAsync(x, cur, bytes, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaEventRecord(op->ev1, s));
  CK(cudaEventSynchronize(op->ev1));
  if (info) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, op->ev0, op->ev1);
    info->status = status;
    info->outer_iters = outer;
    info->inner_iters = inner_total;
    info->restarts = restarts;
    info->fallbacks = fallbacks;
    info->fp64_retries = retries;
    info->true_rel_residual = R;
    info->scaled_rel_residual = scaled;
    info->seconds = ms * 1e-3;
    info->kernel_launches = op->launches;
  }
  return status;
}

}  // extern "C"

namespace {
// Time one precision's column kernels in every valid variant on the operator's
// own arrays (work vectors zeroed; a control block set to "running" before
// each launch) and keep the fastest Thomas and stencil variants.
// The variant the autotuner keeps: the fastest in its trials, unless the
// default variant (dflt >= 0) is within 2% of it.  Variants that close differ
// by less than the run-to-run noise of the trials, the isolated trials do not
// see how the kernels of one iteration share L2, and the dot products'
// rounding order (hence the Krylov iteration count) follows the launch shape:
// keeping the default then keeps the choice, and the solve, the same from run
// to run.
constexpr double kTuneTie = 0.02;
int pick_variant(const std::vector<double>& ms, int dflt) {
  int best = -1;
  for (size_t id = 0; id < ms.size(); ++id)
    if (ms[id] >= 0.0 && (best < 0 || ms[id] < ms[best])) best = (int)id;
  if (best >= 0 && dflt >= 0 && dflt < (int)ms.size() && ms[dflt] >= 0.0 && ms[dflt] <= ms[best] * (1.0 + kTuneTie))
    return dflt;
  return best;
}

template <typename T>
int autotune_prec(hz_op op, int reps, double* best_ms) {
  const int pr = sizeof(T) == 8 ? 1 : 0;
  const Bands<T> a = bands_of<T>(op);
  const Vecs<T>& w = vecs_of<T>(op);
  CK(cudaMemsetAsync(w.rhs, 0, sizeof(T) * 10 * pad64(op->g.n), op->stream));
  Ctl* cfg = op->cfg_h;
  memset(cfg, 0, sizeof(Ctl));
  cfg->state = ST_RUNNING;
  cfg->rsel = 1;
  cfg->r0sel = 1;
  cfg->xzero = 1;
  cfg->alpha = cfg->omega = cfg->beta = 0.5;
  cfg->rho = 1.0;
  cfg->stop2 = -1.0;
  cfg->maxit = 1 << 30;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_it = [&](auto&& launch) -> double {
    double tot = 0.0;
    for (int r = 0; r <= reps; ++r) {  // first launch is a warm-up
      if (cudaMemcpyAsync(op->ctl, cfg, sizeof(Ctl), cudaMemcpyHostToDevice, op->stream) != cudaSuccess) return -1.0;
      cudaEventRecord(e0, op->stream);
      if (launch() != cudaSuccess) return -1.0;
      cudaEventRecord(e1, op->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) tot += ms;
    }
    return tot / reps;
  };
  for (int kind = 0; kind < 2; ++kind) {
    std::vector<double> times(num_variants(pr, kind), -1.0);  // -1: not valid for this grid
    for (int id = 0; id < num_variants(pr, kind); ++id) {
      if (!variant_ok(pr, kind, id, op->g)) continue;
      Launch L = op->L;
      (kind == 0 ? L.vpre : L.vmv)[pr] = id;
      double m1, m2;
      if (kind == 0) {
        m1 = time_it([&] { return launch_pre_p<T>(op->g, a, w, op->ctl, op->red, L); });
        m2 = time_it([&] { return launch_pre_s<T>(op->g, a, w, op->ctl, op->red, L); });
      } else {
        m1 = time_it([&] { return launch_mv_v<T>(op->g, a, w, op->ctl, op->red, L); });
        m2 = time_it([&] { return launch_mv_t<T>(op->g, a, w, op->ctl, op->red, L); });
      }
      const double ms = (m1 < 0 || m2 < 0) ? -1.0 : m1 + m2;  // a failed launch fails the tuning
      if (ms < 0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        set_err(cudaGetLastError(), "autotune launch", __LINE__);
        return HZ_ERR_CUDA;
      }
      times[id] = ms;
    }
    const int best = pick_variant(times, default_variant(pr, kind, op->g.nx));
    if (best >= 0) (kind == 0 ? op->L.vpre : op->L.vmv)[pr] = best;
    if (best_ms) best_ms[kind] = best >= 0 ? times[best] : 1e30;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return HZ_OK;
}

// The tri-SOR kernels of one precision in every variant, on the operator's
// compact arrays (work vectors zeroed, control block "running" before each
// launch): a colour pass with neighbours and an old iterate, both matvecs,
// both first-pass kernels.
template <typename T>
int autotune_sor(hz_op op, int reps) {
  const int pr = sizeof(T) == 8 ? 1 : 0;
  CKS(ensure_sor<T>(op));
  const Bands<T> a = bands_rb<T>(op);
  const Vecs<T>& w = vecs_of<T>(op);
  CK(cudaMemsetAsync(w.rhs, 0, sizeof(T) * 10 * pad64(op->g.n), op->stream));
  Ctl* cfg = op->cfg_h;
  memset(cfg, 0, sizeof(Ctl));
  cfg->state = ST_RUNNING;
  cfg->rsel = 1;
  cfg->r0sel = 1;
  cfg->xzero = 1;
  cfg->alpha = cfg->omega = cfg->beta = 0.5;
  cfg->rho = 1.0;
  cfg->stop2 = -1.0;
  cfg->maxit = 1 << 30;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto time_it = [&](auto&& launch) -> double {
    double tot = 0.0;
    for (int r = 0; r <= reps; ++r) {  // first launch is a warm-up
      if (cudaMemcpyAsync(op->ctl, cfg, sizeof(Ctl), cudaMemcpyHostToDevice, op->stream) != cudaSuccess) return -1.0;
      cudaEventRecord(e0, op->stream);
      if (launch() != cudaSuccess) return -1.0;
      cudaEventRecord(e1, op->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) tot += ms;
    }
    return tot / reps;
  };
  for (int kind = 0; kind < 3; ++kind) {
    std::vector<double> times(sor_num_variants(pr, kind), -1.0);
    for (int id = 0; id < sor_num_variants(pr, kind); ++id) {
      if (!sor_variant_ok(pr, kind, id, op->g.nx)) continue;
      Launch L = op->L;
      L.vsor[pr][kind] = id;
      double ms;
      if (kind == 0)
        ms = time_it([&] { return launch_sor_pass<T>(op->g, a, w.p, w.ph, w.ph, w.t, 1, 1, 1.5, op->ctl, L); });
      else {
        const double m1 = kind == 1 ? time_it([&] { return launch_mv_rb<T>(op->g, a, w, 0, op->ctl, op->red, L); })
                                    : time_it([&] {
                                        return launch_sor_first<T>(op->g, a, w, w.t, 1.5, 0, op->ctl, op->red, L);
                                      });
        const double m2 = kind == 1 ? time_it([&] { return launch_mv_rb<T>(op->g, a, w, 1, op->ctl, op->red, L); })
                                    : time_it([&] {
                                        return launch_sor_first<T>(op->g, a, w, w.t, 1.5, 1, op->ctl, op->red, L);
                                      });
        ms = (m1 < 0 || m2 < 0) ? -1.0 : m1 + m2;
      }
      if (ms < 0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        set_err(cudaGetLastError(), "autotune launch", __LINE__);
        return HZ_ERR_CUDA;
      }
      times[id] = ms;
    }
    const int best = pick_variant(times, -1);
    if (best >= 0) op->L.vsor[pr][kind] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return HZ_OK;
}
}  // namespace

extern "C" {

int hz_op_autotune(hz_op op, int flags) {
  if (!op) return HZ_ERR_INVALID;
  const int reps = 3;
  double ms[2];
  CKS(autotune_prec<float>(op, reps, ms));
  if (flags & 1) {
    CKS(ensure_w64(op));
    CKS(autotune_prec<double>(op, reps, ms));
  }
  if ((flags & 2) && op->g.nx % 2 == 0) {
    CKS(autotune_sor<float>(op, reps));
    if (flags & 1) CKS(autotune_sor<double>(op, reps));
  }
  // the captured inner loops bake the old launch shapes in: rebuild on next use
  for (auto& gs : op->gs) drop_graph(gs);
  for (auto& gs : op->gs_sor) drop_graph(gs);
  store_tuned(op);
  return HZ_OK;
}

int hz_sor_variant_count(int prec, int kind) {
  if ((prec != HZ_PREC_FP32 && prec != HZ_PREC_FP64) || kind < 0 || kind > 2) return 0;
  return sor_num_variants(prec == HZ_PREC_FP64 ? 1 : 0, kind);
}

int hz_op_get_sor_variant(hz_op op, int prec, int kind, int* id) {
  if (!op || !id || hz_sor_variant_count(prec, kind) == 0) return HZ_ERR_INVALID;
  *id = op->L.vsor[prec == HZ_PREC_FP64 ? 1 : 0][kind];
  return HZ_OK;
}

int hz_op_set_sor_variant(hz_op op, int prec, int kind, int id) {
  if (!op || id < 0 || id >= hz_sor_variant_count(prec, kind)) return HZ_ERR_INVALID;
  if (!sor_variant_ok(prec == HZ_PREC_FP64 ? 1 : 0, kind, id, op->g.nx)) return HZ_ERR_INVALID;
  op->L.vsor[prec == HZ_PREC_FP64 ? 1 : 0][kind] = id;
  for (auto& gs : op->gs_sor) drop_graph(gs);
  return HZ_OK;
}

int hz_op_get_variants(hz_op op, int* pre32, int* mv32, int* pre64, int* mv64) {
  if (!op) return HZ_ERR_INVALID;
  if (pre32) *pre32 = op->L.vpre[0];
  if (mv32) *mv32 = op->L.vmv[0];
  if (pre64) *pre64 = op->L.vpre[1];
  if (mv64) *mv64 = op->L.vmv[1];
  return HZ_OK;
}

int hz_op_set_variants(hz_op op, int pre32, int mv32, int pre64, int mv64) {
  if (!op) return HZ_ERR_INVALID;
  const int v[4] = {pre32, mv32, pre64, mv64};
  for (int q = 0; q < 4; ++q) {
    const int pr = q / 2, kind = q % 2;
    if (v[q] < 0) continue;
    if (v[q] >= num_variants(pr, kind) || !variant_ok(pr, kind, v[q], op->g)) return HZ_ERR_INVALID;
  }
  for (int q = 0; q < 4; ++q) {
    const int pr = q / 2, kind = q % 2;
    if (v[q] >= 0) (kind == 0 ? op->L.vpre : op->L.vmv)[pr] = v[q];
  }
  for (auto& gs : op->gs) {
    if (gs.exec) cudaGraphExecDestroy(gs.exec);
    if (gs.graph) cudaGraphDestroy(gs.graph);
    gs.exec = nullptr;
    gs.graph = nullptr;
  }
  return HZ_OK;
}

int hz_profile_enable(hz_op op, int on) {
  if (!op) return HZ_ERR_INVALID;
  op->prof = on != 0;
  for (int k = 0; k < HZ_NUM_KERNELS; ++k) {
    op->p_launch[k] = 0;
    op->p_ms[k] = 0.0;
    op->p_bytes[k] = 0.0;
  }
  return HZ_OK;
}

int hz_profile_read(hz_op op, int kid, long long* launches, double* ms, double* bytes) {
  if (!op || kid < 0 || kid >= HZ_NUM_KERNELS) return HZ_ERR_INVALID;
  if (launches) *launches = op->p_launch[kid];
  if (ms) *ms = op->p_ms[kid];
  if (bytes) *bytes = op->p_bytes[kid];
  return HZ_OK;
}

const char* hz_kernel_name(int kid) {
  static const char* names[HZ_NUM_KERNELS] = {"k_setup",     "k_residual", "k_pre_p", "k_mv_v",
                                              "k_pre_s",     "k_mv_t",     "k_upd",   "k_sor_first",
                                              "k_sor_pass",  "k_mv_rb",    "k_rb_copy"};
  return (kid >= 0 && kid < HZ_NUM_KERNELS) ? names[kid] : "";
}

int hz_get_history(hz_op op, double* hist, int cap) {
  if (!op || !hist || cap < 0) return -HZ_ERR_INVALID;
  if (!op->hist_d) return 0;
  Ctl c;
  if (cudaMemcpy(&c, op->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess) return -HZ_ERR_CUDA;
  int len = std::min(std::min(c.hist_off + (c.xzero ? 0 : 0), op->hist_cap), cap);
  if (len > 0 && cudaMemcpy(hist, op->hist_d, sizeof(double) * len, cudaMemcpyDeviceToHost) != cudaSuccess)
    return -HZ_ERR_CUDA;
  return len;
}

int hz_matvec(hz_op op, int prec, const void* x, void* y) {
  if (!op || !x || !y) return HZ_ERR_INVALID;
  if (prec == HZ_PREC_FP32)
    CK(launch_matvec_hat<float>(op->g, bands_of<float>(op), (const float*)x, (float*)y, op->L));
  else if (prec == HZ_PREC_FP64)
    CK(launch_matvec_hat<double>(op->g, bands_of<double>(op), (const double*)x, (double*)y, op->L));
  else
    return HZ_ERR_INVALID;
  return HZ_OK;
}

// the bounded-wait error word of the kernels launched without a control block
// (read and cleared; HZ_ERR_TIMEOUT if a wait ran out)
int check_kerr(hz_op op) {
  CK(cudaMemcpyAsync(op->err_h, op->kerr_d, sizeof(int), cudaMemcpyDeviceToHost, op->stream));
  CK(cudaStreamSynchronize(op->stream));
  if (*op->err_h) {
    CK(cudaMemsetAsync(op->kerr_d, 0, sizeof(int), op->stream));
    snprintf(g_err, sizeof(g_err), "a bounded wait of a bulk-copy kernel ran out");
    return HZ_ERR_TIMEOUT;
  }
  return HZ_OK;
}

int hz_precond_apply(hz_op op, int prec, const void* r, void* z) {
  if (!op || !r || !z || r == z) return HZ_ERR_INVALID;
  if (prec == HZ_PREC_FP32 && variant_park_mode(0, op->L.vpre[0]) == kParkBulk) {
    CK(launch_tinv<float>(op->g, bands_of<float>(op), (const float*)r, (float*)z, op->L));
    return check_kerr(op);
  }
  if (prec == HZ_PREC_FP32)
    CK(launch_tinv<float>(op->g, bands_of<float>(op), (const float*)r, (float*)z, op->L));
  else if (prec == HZ_PREC_FP64)
    CK(launch_tinv<double>(op->g, bands_of<double>(op), (const double*)r, (double*)z, op->L));
  else
    return HZ_ERR_INVALID;
  return HZ_OK;
}

}  // extern "C"

namespace {
// gather r into compact order (p), sweeps ping-pong between ph and t, scatter to z
template <typename T>
int trisor_apply(hz_op op, int sweeps, double omega, const T* r, T* z) {
  CKS(ensure_sor<T>(op));
  const Bands<T> a = bands_rb<T>(op);
  const Vecs<T>& w = vecs_of<T>(op);
  const Grid& g = op->g;
  CK(launch_rb_copy<T>(g, r, w.p, 1, op->L));
  T* buf[2];
  buf[sweeps % 2] = w.ph;
  buf[(sweeps + 1) % 2] = w.t;
  for (int sw = 0; sw < sweeps; ++sw) {
    T* zin = buf[sw % 2];
    T* zout = buf[(sw + 1) % 2];
    CK(launch_sor_pass<T>(g, a, w.p, zin, sw > 0 ? zin : nullptr, zout, 0, sw > 0 ? 1 : 0, omega, nullptr, op->L));
    CK(launch_sor_pass<T>(g, a, w.p, zout, sw > 0 ? zin : nullptr, zout, 1, 1, omega, nullptr, op->L));
  }
  CK(launch_rb_copy<T>(g, w.ph, z, 0, op->L));
  return HZ_OK;
}
}  // namespace

extern "C" {

int hz_trisor_apply(hz_op op, int prec, int sweeps, double omega, const void* r, void* z) {
  if (!op || !r || !z || r == z) return HZ_ERR_INVALID;
  if (sweeps < 1 || sweeps > 64 || !(omega > 0.0 && omega < 2.0)) return HZ_ERR_INVALID;
  if (op->g.nx % 2 != 0) return HZ_ERR_UNSUPPORTED;
  if (prec == HZ_PREC_FP32) return trisor_apply<float>(op, sweeps, omega, (const float*)r, (float*)z);
  if (prec == HZ_PREC_FP64) {
    CKS(ensure_w64(op));
    return trisor_apply<double>(op, sweeps, omega, (const double*)r, (double*)z);
  }
  return HZ_ERR_INVALID;
}

int hz_precond_matvec(hz_op op, int prec, const void* p, void* ph, void* v) {
  if (!op || !p || !ph || !v) return HZ_ERR_INVALID;
  if (prec == HZ_PREC_FP32 && variant_park_mode(0, op->L.vpre[0]) == kParkBulk) {
    CK(launch_precond_matvec<float>(op->g, bands_of<float>(op), (const float*)p, (float*)ph, (float*)v, op->L));
    return check_kerr(op);
  }
  if (prec == HZ_PREC_FP32)
    CK(launch_precond_matvec<float>(op->g, bands_of<float>(op), (const float*)p, (float*)ph, (float*)v, op->L));
  else if (prec == HZ_PREC_FP64)
    CK(launch_precond_matvec<double>(op->g, bands_of<double>(op), (const double*)p, (double*)ph, (double*)v,
                                     op->L));
  else
    return HZ_ERR_INVALID;
  return HZ_OK;
}

int hz_residual(hz_op op, const double* b, const double* x, double* r, double* rnorm, double* bnorm) {
  if (!op || !b || !x) return HZ_ERR_INVALID;
  CK(launch_residual<float>(op->g, op->A7, op->invc, b, x, nullptr, nullptr, op->w32.rhs, r, 0, op->ctl, op->red,
                            op->L));
  CK(cudaMemcpyAsync(op->rep_h, op->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, op->stream));
  CK(cudaStreamSynchronize(op->stream));
  if (rnorm) *rnorm = std::sqrt(op->rep_h->res_rr);
  if (bnorm) *bnorm = std::sqrt(op->rep_h->res_bb);
  return HZ_OK;
}

int hz_dot(int prec, int64_t n, const void* x, const void* y, void* stream, double* out) {
  if (n < 0 || !out || (n > 0 && (!x || !y))) return HZ_ERR_INVALID;
  if (prec != HZ_PREC_FP32 && prec != HZ_PREC_FP64) return HZ_ERR_INVALID;
  if (n == 0) {
    *out = 0.0;
    return HZ_OK;
  }
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return HZ_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_dot_mu);
  DotScratch& d = g_dot[dev];
  if (!d.partials) {
    CK(cudaMalloc(&d.partials, sizeof(double) * kMaxGrid));
    CK(cudaMalloc(&d.ticket, sizeof(unsigned)));
    CK(cudaMalloc(&d.out, sizeof(double)));
    CK(cudaMallocHost(&d.out_h, sizeof(double)));
    CK(cudaMemset(d.ticket, 0, sizeof(unsigned)));
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<int64_t>(std::min<int64_t>((int64_t)sms * 8, kMaxGrid), (n + 255) / 256);
  cudaStream_t s = (cudaStream_t)stream;
  Red red{d.partials, d.ticket};
  if (prec == HZ_PREC_FP32)
    CK(launch_dot<float>(n, (const float*)x, (const float*)y, red, d.out, grid, s));
  else
    CK(launch_dot<double>(n, (const double*)x, (const double*)y, red, d.out, grid, s));
  CK(cudaMemcpyAsync(d.out_h, d.out, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *out = *d.out_h;
  return HZ_OK;
}

int hz_op_export(hz_op op, int what, int prec, void* dst) {
  if (!op || !dst) return HZ_ERR_INVALID;
  const int64_t n = op->g.n;
  const void* src = nullptr;
  size_t bytes = 0;
  if (what == 0 && prec == HZ_PREC_FP32) { src = op->ah32; bytes = 6 * n * sizeof(float); }
  else if (what == 0 && prec == HZ_PREC_FP64) { src = op->ah64; bytes = 6 * n * sizeof(double); }
  else if (what == 1 && prec == HZ_PREC_FP32) { src = op->th32; bytes = 3 * n * sizeof(float); }
  else if (what == 1 && prec == HZ_PREC_FP64) { src = op->th64; bytes = 3 * n * sizeof(double); }
  else if (what == 2 && op->hb != HB_F32) {
    for (int b = 0; b < 4; ++b)
      CK(cudaMemcpyAsync((uint16_t*)dst + b * n, op->h16 + b * pad64(n), n * sizeof(uint16_t),
                         cudaMemcpyDeviceToDevice, op->stream));
    CK(cudaStreamSynchronize(op->stream));
    return HZ_OK;
  }
  else return HZ_ERR_INVALID;
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, op->stream));
  CK(cudaStreamSynchronize(op->stream));
  return HZ_OK;
}

int hz_batched_debug(long long timeout_ns, int leave_block) {
  if (timeout_ns <= 0) timeout_ns = 2000000000LL;
  g_batch_timeout_ns = timeout_ns;
  g_batch_leave_block = leave_block;
  return HZ_OK;
}

int hz_batched_set_vec(int vec) {
  if (vec != 0 && vec != 1 && vec != 4) return HZ_ERR_INVALID;
  g_batch_vec = vec;
  return HZ_OK;
}

// batched solves: systems of at least this many points each fill the GPU alone
// (the automatic strategy then solves them one after another)
constexpr int64_t kBatchSeqMinPoints = int64_t(1) << 20;

int hz_solve_batched(int nsys, const hz_op* ops, const double* const* b, const double* const* x0, double* const* x,
                     const hz_solve_params* pp, hz_solve_info* infos) {
  return hz_solve_batched_ex(nsys, ops, b, x0, x, pp, infos, HZ_BATCH_AUTO);
}

int hz_solve_batched_ex(int nsys, const hz_op* ops, const double* const* b, const double* const* x0,
                        double* const* x, const hz_solve_params* pp, hz_solve_info* infos, int strategy) {
  if (nsys < 1 || nsys > kMaxSys || !ops || !b || !x) return HZ_ERR_INVALID;
  if (strategy != HZ_BATCH_AUTO && strategy != HZ_BATCH_PERSISTENT && strategy != HZ_BATCH_SEQUENTIAL)
    return HZ_ERR_INVALID;
  hz_solve_params p;
  if (pp)
    p = *pp;
  else
    hz_default_params(&p);
  if (!(p.tol > 0.0) || p.max_outer < 0 || p.max_inner < 1 || p.restart < 1) return HZ_ERR_INVALID;
  if (p.mode != HZ_MODE_MIXED_IR || p.krylov != HZ_KRYLOV_BICGSTAB || p.precond != HZ_PRE_TRI)
    return HZ_ERR_UNSUPPORTED;
  const double eta = p.inner_tol > 0.0 ? p.inner_tol : 1e-4;
  cudaStream_t s = ops[0] ? ops[0]->stream : nullptr;
  int vec = 4;
  for (int q = 0; q < nsys; ++q) {
    if (!ops[q] || !b[q] || !x[q]) return HZ_ERR_INVALID;
    if (ops[q]->stream != s) return HZ_ERR_INVALID;
    if (!is_device_ptr(b[q]) || !is_device_ptr(x[q]) || (x0 && x0[q] && !is_device_ptr(x0[q])))
      return HZ_ERR_INVALID;
    if (ops[q]->g.nx % 4) vec = 1;
  }
  // Four columns per thread wherever the rows allow it: a phase of the
  // persistent kernel takes about as long as one thread's march down its
  // columns' levels, whatever the number of columns per thread (measured
  // equal per iteration on 64 systems of 48x36x70, 1.6x faster with four on
  // 32 right-hand sides of 192x144x70).
  if (g_batch_vec == 1) vec = 1;
  if (g_batch_vec == 4 && vec != 4) return HZ_ERR_INVALID;
  // Systems that each fill the GPU on their own run one after another through
  // the single-system path (its graph-captured inner loop and per-kernel
  // variants at full occupancy); smaller ones share the persistent launch,
  // one launch for the whole batch, which pays off when a system alone cannot
  // keep the SMs busy.
  if (strategy == HZ_BATCH_AUTO) {
    int64_t smallest = ops[0]->g.n;
    for (int q = 1; q < nsys; ++q) smallest = std::min(smallest, ops[q]->g.n);
    strategy = smallest >= kBatchSeqMinPoints ? HZ_BATCH_SEQUENTIAL : HZ_BATCH_PERSISTENT;
  }
  if (strategy == HZ_BATCH_SEQUENTIAL) {
    int worst = HZ_OK;
    for (int q = 0; q < nsys; ++q) {
      hz_solve_info tmp;
      const int st = hz_solve(ops[q], b[q], x0 ? x0[q] : nullptr, x[q], &p, infos ? &infos[q] : &tmp);
      if (st != HZ_OK && (worst == HZ_OK || st == HZ_ERR_CUDA)) worst = st;
      if (st == HZ_ERR_CUDA) return st;
    }
    return worst;
  }
  // the whole solve of every system in one persistent launch (refinement loop
  // on the device), replayed from a captured graph when params->use_graph is
  // set and the same systems come again
  std::vector<SysDesc> sys(nsys);
  std::vector<int> occ(nsys, 0);
  int64_t item0 = 0;
  for (int q = 0; q < nsys; ++q) {
    hz_op op = ops[q];
    for (int r = 0; r < q; ++r)
      if (ops[r] == op) ++occ[q];
    Vecs<float> w = op->w32;
    Ctl* ctl = op->ctl;
    double* xb = op->xscr;
    if (occ[q] > 0) {  // a further right-hand side of this operator: its own work vectors
      if ((int)op->rhs_ws.size() < occ[q]) op->rhs_ws.resize(occ[q]);
      hz_op_s::RhsWs& rw = op->rhs_ws[occ[q] - 1];
      if (!rw.base) {
        float* base = nullptr;
        Ctl* c = nullptr;
        double* x2 = nullptr;
        cudaError_t e = cudaMalloc(&base, sizeof(float) * 10 * (size_t)pad64(op->g.n));
        if (e == cudaSuccess) e = cudaMalloc(&c, sizeof(Ctl));
        if (e == cudaSuccess) e = cudaMalloc(&x2, sizeof(double) * (size_t)op->g.n);
        if (e != cudaSuccess) {
          if (base) cudaFree(base);
          if (c) cudaFree(c);
          set_err(e, "cudaMalloc (batched right-hand side)", __LINE__);
          return e == cudaErrorMemoryAllocation ? HZ_ERR_OOM : HZ_ERR_CUDA;
        }
        rw.base = base;
        rw.w = carve(base, op->g.n);
        rw.ctl = c;
        rw.xb = x2;
      }
      w = rw.w;
      ctl = rw.ctl;
      xb = rw.xb;
    }
    const int64_t ni = (op->g.ncol / vec + kBS - 1) / kBS;
    SysDesc d{};
    d.g = op->g;
    d.a = bands_of<float>(op, false);
    d.w = w;
    d.ctl = ctl;
    d.item0 = item0;
    d.nitems = ni;
    d.A7 = op->A7;
    d.invc = op->invc;
    d.b = b[q];
    d.x0 = (x0 && x0[q]) ? x0[q] : nullptr;
    d.xa = x[q];
    d.xb = xb;
    sys[q] = d;
    item0 += ni;
  }
  hz_op o0 = ops[0];
  std::vector<Ctl> cfg(nsys);
  for (int q = 0; q < nsys; ++q) {
    Ctl& c = cfg[q];
    memset(&c, 0, sizeof(Ctl));
    c.eta = eta;
    c.maxit = p.max_inner;
    c.restart_every = p.restart;
    c.body_limit = 4 * p.max_inner + 64;
    c.xzero = 1;
    c.xz = 1;
    c.state = ST_CONVERGED;
    c.tol = p.tol;
    c.max_outer = p.max_outer;
  }
  CK(cudaEventRecord(o0->ev0, s));
  for (int q = 0; q < nsys; ++q) CK(cudaMemcpyAsync(sys[q].ctl, &cfg[q], sizeof(Ctl), cudaMemcpyHostToDevice, s));
  // loop bound of the persistent kernel: every refinement step's inner solve and its residual pass
  const int max_loops = (p.max_outer + 1) * (p.max_inner + 8) + 8;
  int* err_h = &o0->err_h[0];
  *err_h = 0;
  CK(launch_batched(sys.data(), nsys, vec, max_loops, g_batch_timeout_ns, g_batch_leave_block, s, err_h, o0->sms,
                    p.use_graph != 0));
  for (int q = 0; q < nsys; ++q) CK(cudaMemcpyAsync(&cfg[q], sys[q].ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(o0->ev1, s));
  CK(cudaEventSynchronize(o0->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, o0->ev0, o0->ev1);
  int worst = HZ_OK;
  if (*err_h) {
    snprintf(g_err, sizeof(g_err), "batched solve: a grid-barrier wait exceeded %lld ns", g_batch_timeout_ns);
    worst = HZ_ERR_TIMEOUT;
  }
  for (int q = 0; q < nsys; ++q) {
    const Ctl& c = cfg[q];
    int st = *err_h ? HZ_ERR_TIMEOUT : (c.odone ? c.ostatus : HZ_ERR_NOT_CONVERGED);
    if (st != HZ_OK && worst == HZ_OK) worst = st;
    if (infos) {
      infos[q].status = st;
      infos[q].outer_iters = c.outer;
      infos[q].inner_iters = c.inner_total;
      infos[q].restarts = c.restart_total;
      infos[q].fallbacks = 0;
      infos[q].fp64_retries = 0;
      infos[q].true_rel_residual = c.R;
      infos[q].scaled_rel_residual = c.last_bnorm2 > 0.0 ? std::sqrt(c.last_rnorm2 / c.last_bnorm2) : 0.0;
      infos[q].seconds = ms * 1e-3;
      infos[q].kernel_launches = 1;
    }
  }
  return worst;
}

}  // extern "C"
