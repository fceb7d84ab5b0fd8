// hz_internal.cuh -- shared definitions of the CUDA path (device control block,
// reductions, launch wrappers).  Everything here belongs to the GPU library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hz.h"

namespace hz {

constexpr int kBS = 128;          // threads per block of the column kernels
constexpr int kMaxND = 4;         // dots reduced by one launch at most
constexpr int kMaxGrid = 8192;    // partial-sum slots per reduction buffer

struct Grid {
  int nx, ny, nz;
  int64_t ncol, n;
};

// Inner Krylov state machine (lives in device memory; each kernel reads it at
// entry and the last block of a reduction writes it).
enum State : int {
  ST_RUNNING = 0,
  ST_CONVERGED = 1,
  ST_MAXIT = 2,
  ST_NONFINITE = 3,
  ST_RESTART = 4,
  ST_HALF = 5,  // ||s|| met the tolerance: finish with x += alpha ph
};

struct Ctl {
  // BiCGStab scalars, FP64 (the paper's 64-bit global sums, Sec. 4)
  double rho, alpha, omega, beta;
  double bnorm2;   // ||rhs||^2 of the inner system
  double stop2;    // (eta ||rhs||)^2
  double rnorm2, r0norm2, snorm2;
  int iter, since, restarts, state;
  int maxit, restart_every;
  int fresh;   // 1: next p = r (start or restart)
  int rsel;    // 0: r still equals rhs (read rhs); 1: r buffer valid
  int r0sel;   // 0: r0 = rhs; 1: r0 buffer
  int xzero;   // 1: x not yet written (= 0)
  int hist_cap;
  int pad0;
  double* hist;  // recursive relative residual per iteration (may be null)
  // outer true-residual results (written by the residual kernel)
  double res_rr, res_bb, res_hh;
  double eta;
  // report of the inner solve that the residual kernel consumed
  double last_rnorm2, last_bnorm2;
  int last_iter, last_restarts, last_state, hist_off;
  // bodies of the inner loop launched since the last residual pass, and the
  // hard limit after which the loop stops whatever the state says
  int bodies, body_limit;
  // the paper's mixed-precision solver (Sec. 3): the inner iterate x kept in
  // FP64 here while every other vector is FP32 (null: x is the FP32 vector)
  double* x64;
  // 1: dot products summed in FP32 at every level, thread, block and grid (the
  // paper's original 32-bit global sums, Sec. 4); 0: FP64 across threads
  int dot32;
  // device error word of the inner solve (bit 0: a bounded wait of a
  // bulk-copy kernel ran out); the host reports HZ_ERR_TIMEOUT
  int kerr;
  // the refinement loop of the batched solver, run on the device: target,
  // ||b||^2, R before the last step, the last R; steps taken, the limit,
  // stalls in a row, done flag and final status, the buffer holding x (0: xa,
  // 1: xb), x still zero, and the totals of the inner solves
  double tol, ob, Rprev, R;
  int outer, max_outer, stall, odone, ostatus, cur, xz, inner_total, restart_total, pad2;
};

struct Red {
  double* partials;  // kMaxGrid * kMaxND
  unsigned* ticket;
};

template <typename T>
struct Bands {  // scaled operator in one precision, Ahat = I + bands
  const T *E, *W, *N, *S, *U, *D;
  const T *m, *l, *cp;  // Thomas factors of T (unit diagonal)
  // 16-bit copies of the horizontal bands (E, W, N, S at h16 + b * h16s), read
  // instead of E..S by the FP32 stencil kernels when h16fmt is HB_BF16 or HB_FP16
  const uint16_t* h16;
  int64_t h16s;
  int h16fmt;
};

// storage of the horizontal bands read by the FP32 stencil kernels
enum HBand : int { HB_F32 = 0, HB_BF16 = 1, HB_FP16 = 2 };

template <typename T>
struct Vecs {  // inner Krylov vectors
  T *rhs, *r, *r0, *p, *ph, *v, *s, *sh, *t, *x;
};

// Running sum of a dot product's per-batch partials within one thread.  FP32:
// an unevaluated pair hi + lo updated by Knuth's TwoSum (error-free in
// round-to-nearest, Knuth, TAOCP vol. 2, Sec. 4.2.2), which carries about 48
// significant bits with FP32 additions only, so the loop issues no FP64
// instruction (FP64 issue is scarce on this GPU and a per-batch FP64 add
// stalls every warp at the batch boundary).  The thread's total is read once,
// in FP64, by the grid reduction.  FP64: a plain double.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<float> {
  float hi, lo;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bv = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(x, bv));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
  // f32: the plain FP32 running sum (hi alone is exactly what repeated FP32
  // additions give; lo only carries their rounding errors)
  __device__ __forceinline__ double total(bool f32) const { return f32 ? (double)hi : value(); }
};
template <>
struct DotAcc<double> {
  double s;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ double total(bool) const { return s; }
};

// acc + x with the sum rounded to FP32 when f32 (an FP32 accumulator held in a double)
__device__ __forceinline__ double acc_add(double acc, double x, bool f32) {
  return f32 ? (double)__fadd_rn((float)acc, (float)x) : acc + x;
}

// Deterministic block + grid reduction of ND doubles.  Every block stores its
// partial in a fixed slot; the last block to arrive (ticket) sums the slots in
// slot order, so the result depends only on the launch shape.  Returns true in
// thread 0 of the last block, with the totals in out.  f32: every addition of
// the reduction is rounded to FP32 (the inputs are taken as FP32 values): the
// all-32-bit global sums of the paper's first mixed-precision solver (Sec. 4).
template <int ND>
__device__ __forceinline__ bool grid_reduce(double (&v)[ND], const Red& red, double (&out)[ND], bool f32 = false) {
  __shared__ double sm[ND][32];
  __shared__ int amlast;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  auto warp_sum = [&](double x) -> double {
    if (f32) {
      float xf = (float)x;
#pragma unroll
      for (int o = 16; o; o >>= 1) xf = __fadd_rn(xf, __shfl_xor_sync(0xffffffffu, xf, o));
      return (double)xf;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    const double x = warp_sum(v[d]);
    if (lane == 0) sm[d][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const double x = warp_sum(lane < nw ? sm[d][lane] : 0.0);
      if (lane == 0) red.partials[(size_t)blockIdx.x * ND + d] = x;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned t = atomicAdd(red.ticket, 1u);
    amlast = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!amlast) return false;
  __threadfence();
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    double x = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      x = acc_add(x, __ldcg(&red.partials[(size_t)b * ND + d]), f32);
    v[d] = warp_sum(x);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int d = 0; d < ND; ++d) sm[d][warp] = v[d];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      double x = 0.0;
      for (int w = 0; w < nw; ++w) x = acc_add(x, sm[d][w], f32);
      out[d] = x;
    }
    *red.ticket = 0u;
    return true;
  }
  return false;
}

// ---- launch wrappers (defined in the kernel translation units) ----
struct Launch {
  int sms;           // SMs of the device
  int64_t wcol;      // blocks needed to give every column its own thread (kBS per block)
  int64_t wflat;     // blocks of 256 threads needed by the elementwise kernels
  cudaStream_t stream;
  int vpre[2];       // variant of the Thomas kernels, [0] FP32, [1] FP64
  int vmv[2];        // variant of the stencil kernels
  int vsor[2][3];    // tri-SOR variants: [prec][0 colour pass, 1 matvec, 2 first pass]
  int nz;            // levels of the operator (shared-memory size of the parking variants)
  int* err;          // device error word of launches without a control block (bounded waits)
};

// tri-SOR kernel variants (kind 0 colour pass, 1 matvec, 2 first pass):
// vec = columns per thread (must divide nx/2), depth = levels per
// software-pipelined batch, minb = launch bound in blocks of kBS threads per
// SM (registers per thread = 65536 / (kBS * minb))
int sor_num_variants(int prec, int kind);
void sor_variant_shape(int prec, int kind, int id, int* vec, int* depth, int* minb);
bool sor_variant_ok(int prec, int kind, int id, int nx);

// Column-kernel variants: kind 0 = Thomas (k_pre_p, k_pre_s), kind 1 = stencil
// (k_mv); prec 0 = FP32, 1 = FP64.  vec = columns per thread (must divide nx),
// depth = levels per software-pipelined batch.
int num_variants(int prec, int kind);
void variant_shape(int prec, int kind, int id, int* vec, int* depth);
// the Thomas variant parks its forward sweep in shared memory (nz * kBS * vec values per block)
bool variant_parks_smem(int prec, int kind, int id);
// where Thomas variant id parks its forward sweep (0 output vector, 1 shared memory, 2 output vector with L2 priorities)
int variant_park_mode(int prec, int id);
template <typename T>
void warm_kernels(const Launch& L);

// ---- the bulk-copy Thomas kernels (hz_thomas_bulk.cu), FP32 ----
constexpr int kParkBulk = 3;  // their park mode in the Thomas variant tables (PARK_BULK)
// mode 0: k_pre_p's work (p update + T^-1), 1: k_pre_s's (s = r - alpha v + T^-1),
// 2: z = T^-1 r alone.  Valid when ncol % 4 == 0 and the tile's parked sweep fits.
bool thomas_bulk_ok(const Grid& g);
// stages: ring slots, 3, 4 or 5
cudaError_t launch_thomas_bulk(int mode, int stages, int per_sm_cap, const Grid& g, const Bands<float>& a,
                               const Vecs<float>& w, const float* r, float* z, Ctl* ctl, int* err, const Launch& L);
void warm_thomas_bulk(const Launch& L, int nz);

// Blocks for a grid-stride kernel: every SM filled to that kernel's own
// occupancy (queried once per kernel and cached) or to per_sm_cap blocks when
// that is smaller and positive, capped by the work and by the slots of the
// reduction buffer.  warm_launch_cache() queries every kernel up front so that
// no query happens during stream capture.
int grid_for(const void* kernel, int block, const Launch& L, int64_t work_blocks, size_t smem = 0,
             int per_sm_cap = 0);
void warm_launch_cache(const Launch& L);

template <typename T>
cudaError_t launch_pre_p(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L);
template <typename T>
cudaError_t launch_mv_v(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L);
template <typename T>
cudaError_t launch_pre_s(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L);
template <typename T>
cudaError_t launch_mv_t(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L);
template <typename T>
cudaError_t launch_upd(const Grid& g, const Vecs<T>& w, Ctl* ctl, Red red, unsigned long long cond, int use_cond,
                       const Launch& L);

// building blocks for the kernel-level entry points
template <typename T>
cudaError_t launch_matvec_hat(const Grid& g, const Bands<T>& a, const T* x, T* y, const Launch& L);
template <typename T>
cudaError_t launch_tinv(const Grid& g, const Bands<T>& a, const T* r, T* z, const Launch& L);
template <typename T>
cudaError_t launch_precond_matvec(const Grid& g, const Bands<T>& a, const T* p, T* ph, T* v, const Launch& L);

// ---- tri-SOR preconditioner in colour-compact column order (hz_sor.cu) ----
// compact column of (i, j): ((i + j) & 1) * ncol/2 + j * nx/2 + i/2 (nx even).
// Bands and vectors passed to these are all in compact order.
template <typename T>
cudaError_t launch_rb_copy(const Grid& g, const T* src, T* dst, int to_compact, const Launch& L);
// mode 0: p update (with start/restart handling), mode 1: s = r - alpha v; then
// z1 = omega T^-1 (p or s) on the red half (the first sweep's red pass)
template <typename T>
cudaError_t launch_sor_first(const Grid& g, const Bands<T>& a, const Vecs<T>& w, T* z1, double omega, int mode,
                             Ctl* ctl, Red red, const Launch& L);
// zout(colour) = (1 - omega) zold + omega T^-1 (rc - H znbr); zold may be null (zero), nbr = 0: znbr is zero
template <typename T>
cudaError_t launch_sor_pass(const Grid& g, const Bands<T>& a, const T* rc, const T* znbr, const T* zold, T* zout,
                            int colour, int nbr, double omega, const Ctl* ctl, const Launch& L);
// mode 0: v = Ahat ph, <r0, v> -> alpha; mode 1: t = Ahat sh, <t, s>, <t, t> -> omega
template <typename T>
cudaError_t launch_mv_rb(const Grid& g, const Bands<T>& a, const Vecs<T>& w, int mode, Ctl* ctl, Red red,
                         const Launch& L);
template <typename T>
void warm_sor(const Launch& L);
template <typename T>
cudaError_t launch_dot(int64_t n, const T* x, const T* y, Red red, double* out_dev, int grid, cudaStream_t s);

// operator setup and the FP64 true residual (hz_setup.cu)
struct SetupOut {
  float* ah32;    // [6][n]
  float* th32;    // [3][n]
  double* ah64;   // [6][n]
  double* th64;   // [3][n]
  double* invc;   // [n]
  int* err;       // device error word
};
cudaError_t launch_setup(const Grid& g, const double* A7, SetupOut o, const Launch& L);
// 16-bit copies (fmt HB_BF16 or HB_FP16) of the horizontal bands E, W, N, S of
// the FP64 scaled operator ah64 ([6][n]): out[b * stride + p], rounded to
// nearest even (BF16: from the FP32 rounding of the value, FP16: directly)
cudaError_t launch_h16(const Grid& g, const double* ah64, uint16_t* out, int64_t stride, int fmt, const Launch& L);

// residual modes
enum ResMode : int { RES_ZERO = 0, RES_X0 = 1, RES_UPDATE = 2, RES_FROM_DELTA = 3 };
// r = b - A x (FP64); x per mode; writes x (modes X0 with x!=x0, UPDATE, FROM_DELTA),
// rhs_out = D^-1 r in float or double, r_out (may be null); reduces ||r||^2, ||b||^2,
// ||rhs||^2 and prepares ctl for the next inner solve with tolerance eta.
template <typename D>
cudaError_t launch_residual(const Grid& g, const double* A7, const double* invc, const double* b, const double* x0,
                            double* x, const D* delta, D* rhs_out, double* r_out, int mode, Ctl* ctl, Red red,
                            const Launch& L);
// the same with an FP64 correction and an FP32 right-hand side (the paper's
// mixed-precision solver keeps its inner iterate in FP64)
cudaError_t launch_residual_x64(const Grid& g, const double* A7, const double* invc, const double* b,
                                const double* xin, double* xout, const double* delta, float* rhs, Ctl* ctl, Red red,
                                const Launch& L);

// ---- flexible GMRES (hz_fgmres.cu) ----
constexpr int kMaxFgm = 64;  // largest restart length
struct FgmState {            // small dense state of FGMRES, FP64, device memory
  double H[(kMaxFgm + 1) * kMaxFgm];  // Hessenberg, column-major, then R after the rotations
  double cs[kMaxFgm], sn[kMaxFgm], g[kMaxFgm + 1], y[kMaxFgm];
  double h1[kMaxFgm + 1], h2[kMaxFgm + 1];  // the two Gram-Schmidt passes
  double wn2, beta, resid, wnorm, r2;
};
struct FgmWs {
  int m = 0;
  float* base = nullptr;    // V_0..V_m, Z_0..Z_(m-1), w: (2m+2) vectors
  float** vptr = nullptr;   // device array of those 2m+1 vector pointers (V then Z)
  float* w = nullptr;
  double* part = nullptr;   // [grid][kMaxFgm+1] partial sums
  FgmState* st = nullptr;   // device
};
cudaError_t fgm_multidot(const FgmWs& W, int64_t n, float* const* Vdev, int nv, const float* w, double* dst,
                         const Launch& L);
cudaError_t fgm_update(const FgmWs& W, int64_t n, float* const* Vdev, int nv, const double* c, float* w,
                       double* nrm2_dst, const Launch& L);
cudaError_t fgm_scale(int64_t n, const float* x, float* y, const double* s, int inv_sqrt, const Launch& L);
cudaError_t fgm_step(FgmState* st, int j, cudaStream_t s);
cudaError_t fgm_solve_update(FgmState* st, int64_t n, float* const* Zdev, int k, float* x, int xzero,
                             const Launch& L);
cudaError_t fgm_start(FgmState* st, const double* nrm2, cudaStream_t s);
cudaError_t fgm_residual(const FgmWs& W, const Grid& g, const Bands<float>& a, const float* rhs, const float* x,
                         float* r, double* nrm2_dst, const Launch& L);

// ---- learned stage (hz_nn.cu) ----
// z <- z + sigma * NN(e1 / sigma), sigma = sqrt(*nrm2 / n), on a full (periodic) field
int nn_stage_apply(hz_nn_s* nn, const Grid& g, const float* e1, const double* nrm2, float* z, cudaStream_t s);
// waits for the network's stream and reports HZ_ERR_TIMEOUT if a tensor-core
// kernel's bounded wait gave up since the last check
int nn_stage_status(hz_nn_s* nn, cudaStream_t s);
// training-pair helpers: stage 0: rs = r / A_C, e = xs - xk; stage 1: in = e1 / sigma, tg = (e - z1) / sigma
cudaError_t nn_pair_launch(int64_t n, const double* A7, const double* b, const double* xk, const double* xs,
                           const double* r, float* rs, float* e, const float* e1, const float* z1, const double* nrm2,
                           float* in, float* tg, int stage, cudaStream_t s);

// ---- batched persistent solve (hz_batched.cu) ----
constexpr int kMaxSys = 64;
struct SysDesc {
  Grid g;
  Bands<float> a;
  Vecs<float> w;
  Ctl* ctl;
  int64_t item0;   // first global work item of this system (item = kBS column groups)
  int64_t nitems;  // items of this system
  // the stencil and update phases (no vertical coupling) also split the levels:
  // level item = (chunk of lchunk levels, column item); set by launch_batched
  int64_t litem0;  // first global level item of this system
  int lchunk;      // levels per chunk
  int nchunk;      // chunks (nitems * nchunk level items)
  // the system's refinement loop: unscaled FP64 bands [7][n], 1/A_C, b, the
  // initial guess (null: zero), the caller's x (where the result ends) and a
  // second buffer for the ping-pong of x
  const double* A7;
  const double* invc;
  const double* b;
  const double* x0;
  double* xa;
  double* xb;
};
// Runs the whole mixed-precision solve of nsys systems -- FP64 residuals,
// FP32 inner BiCGStab, refinement updates and the per-system decisions on tol,
// max_outer and stagnation -- in one cooperative launch on `stream`; each
// control block must hold the configuration (eta, maxit, restart, tol,
// max_outer).  *err_h (pinned host) receives the device error word (bit 0: a
// grid-barrier wait exceeded timeout_ns) once the stream reaches it; the call
// does not wait.  vec = 4 needs nx % 4 == 0 for every system, else pass 1.
// leave_block >= 0 makes that block leave after its first barrier (test hook
// for the bounded wait).  graph: capture the launch once into a CUDA graph
// and replay it while the systems (the SysDesc array) stay the same.
cudaError_t launch_batched(const SysDesc* sys_h, int nsys, int vec, int max_loops, long long timeout_ns,
                           int leave_block, cudaStream_t stream, int* err_h, int sms, bool graph);

}  // namespace hz
