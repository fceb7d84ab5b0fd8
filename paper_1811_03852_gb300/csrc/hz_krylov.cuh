// hz_krylov.cuh -- the inner BiCGStab iteration on sm_103a (kernel templates;
// instantiated for FP32 in hz_krylov_f32.cu and for FP64 in hz_krylov_f64.cu).
//
// Right-preconditioned ("post-conditioned", Maynard & Walters Sec. 2)
// BiCGStab (van der Vorst 1992) on Ahat y = rhs with C = T^-1.  Every scalar
// lives in the device control block, so the loop needs no host round trip
// and runs as a CUDA-graph while loop.  One iteration:
//
//   k_pre_start : first iteration after a start (p = r) or a restart (Sec. 4)
//   k_pre_p     : p = r + beta (p - omega v)         then ph = T^-1 p    (Thomas along k)
//   k_mv<0>     : v = p + H ph,  <r0, v>  -> alpha   (T ph = p, so Ahat ph = p + H ph)
//   k_pre_s     : s = r - alpha v                    then sh = T^-1 s
//   k_mv<1>     : t = s + H sh,  <t, s>, <t, t>, <s, s> -> half-step exit test, omega
//   k_upd       : x += alpha ph + omega sh, r = s - omega t, <r0, r>, <r, r> -> beta, stop/restart
//
// H = the four horizontal bands (E, W, N, S) of Ahat.  Column kernels come in
// variants (vector width V columns per thread, U levels per software-pipelined
// batch) chosen per operator by hz_op_autotune.  Partial sums are FP32 (FP64
// in the FP64 solver) over at most one batch and FP64 across batches, threads
// and blocks (the paper's 64-bit global sums, Sec. 4); the grid reduction is
// deterministic for a given variant (fixed slots summed in slot order).
#pragma once

#include <type_traits>

#include "hz_columns.cuh"

namespace hz {

// ---- variants ----------------------------------------------------------------
template <typename T>
struct Variants;
// Thomas variants: V columns per thread, U levels per batch, pre_p where the
// forward sweep is parked (ParkMode: 0 the output vector, 1 shared memory,
// nz * kBS * V values per block, 2 the output vector with L2 priorities, 3 the
// bulk-copy kernel of hz_thomas_bulk.cu: four columns per thread, U = its ring
// slots) and
// pre_b resident blocks per SM (0: as many as fit).  Fewer resident columns
// keep the parked sweep of every column in flight inside L2.  Stencil
// variants: mv_v columns per thread, mv_u levels per batch, mv_h L2 priorities
// (the arrays read once evict-first, so that rows of x stay in L2), mv_b
// resident blocks per SM (0: as many as fit; fewer rows in flight keep the
// north/south neighbour rows of x in L2 until they are re-read).
template <>
struct Variants<float> {
  static constexpr int NPRE = 18, NMV = 11;
  static constexpr int pre_v[NPRE] = {1, 4, 4, 2, 1, 1, 2, 2, 4, 2, 2, 4, 2, 4, 4, 4, 4, 4};
  static constexpr int pre_u[NPRE] = {8, 2, 1, 4, 8, 4, 4, 2, 2, 4, 4, 2, 4, 5, 3, 4, 5, 8};
  static constexpr int pre_p[NPRE] = {0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 3};
  static constexpr int pre_b[NPRE] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 4, 0, 0, 3, 0, 0, 0, 1, 1};
  static constexpr int mv_v[NMV] = {1, 4, 2, 2, 4, 2, 2, 4, 4, 4, 2};
  static constexpr int mv_u[NMV] = {4, 1, 2, 1, 1, 2, 1, 1, 1, 1, 2};
  static constexpr int mv_h[NMV] = {0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1};
  static constexpr int mv_b[NMV] = {0, 0, 0, 0, 0, 0, 0, 4, 3, 5, 4};
};
template <>
struct Variants<double> {
  static constexpr int NPRE = 6, NMV = 5;
  static constexpr int pre_v[NPRE] = {1, 2, 2, 2, 2, 1};
  static constexpr int pre_u[NPRE] = {4, 2, 1, 1, 1, 4};
  static constexpr int pre_p[NPRE] = {0, 0, 0, 2, 2, 2};
  static constexpr int pre_b[NPRE] = {0, 0, 0, 3, 0, 0};
  static constexpr int mv_v[NMV] = {1, 2, 1, 2, 1};
  static constexpr int mv_u[NMV] = {2, 1, 1, 1, 2};
  static constexpr int mv_h[NMV] = {0, 0, 0, 1, 1};
  static constexpr int mv_b[NMV] = {0, 0, 0, 0, 0};
};

constexpr int kMinBlocks = 6;  // launch bound of the column kernels: at most 80 registers per thread

// shared memory of a parking variant for nz levels (0 for the others), and its
// limit (below the 227 KB opt-in maximum, which also holds the kernels' static
// reduction buffers)
constexpr size_t kParkMax = 200 * 1024;
template <typename T, int V, int P>
constexpr size_t park_bytes(int nz) {
  return P == PARK_SMEM ? (size_t)nz * kBS * V * sizeof(T) : 0;
}

template <typename T>
__device__ __forceinline__ T ldro(const T* p) {
  return __ldg(p);
}

struct ColNbr {
  int64_t ie, iw;  // offsets of the east / west neighbour (periodic)
  bool hn, hs;     // north / south neighbour exists
};

__device__ __forceinline__ ColNbr col_nbr(const Grid& g, int64_t col) {
  const int i = (int)(col % g.nx);
  const int j = (int)(col / g.nx);
  ColNbr c;
  c.ie = (i == g.nx - 1) ? -(int64_t)(g.nx - 1) : 1;
  c.iw = (i == 0) ? (int64_t)(g.nx - 1) : -1;
  c.hn = j + 1 < g.ny;
  c.hs = j > 0;
  return c;
}

// (Ahat x)_idx with all six bands (restart and the test entry point); x may be
// stored in FP64 while the arithmetic is T's (the paper's mixed-precision solver)
// horizontal band b at idx as the stencil kernels read it (16-bit copy if any)
template <typename T>
__device__ __forceinline__ T hband(const Bands<T>& a, int b, int64_t idx) {
  if (sizeof(T) == 4 && a.h16fmt != HB_F32) return (T)widen16(a.h16[(int64_t)b * a.h16s + idx], a.h16fmt);
  const T* base = b == 0 ? a.E : b == 1 ? a.W : b == 2 ? a.N : a.S;
  return base[idx];
}

template <typename T, typename X>
__device__ __forceinline__ T ahat_point(const Grid& g, const Bands<T>& a, const X* __restrict__ x, int64_t idx, int k,
                                        const ColNbr& c) {
  T y = (T)x[idx];
  y = fma(hband(a, 0, idx), (T)x[idx + c.ie], y);
  y = fma(hband(a, 1, idx), (T)x[idx + c.iw], y);
  if (c.hn) y = fma(hband(a, 2, idx), (T)x[idx + g.nx], y);
  if (c.hs) y = fma(hband(a, 3, idx), (T)x[idx - g.nx], y);
  if (k + 1 < g.nz) y = fma(a.U[idx], (T)x[idx + g.ncol], y);
  if (k > 0) y = fma(a.D[idx], (T)x[idx - g.ncol], y);
  return y;
}

// ---- control steps (run by one thread once a reduction is complete; shared by
// the single-system kernels and the batched persistent kernel) ----------------
// restart (Sec. 4): rr = ||r||^2 of the recomputed residual, r0 = r
__device__ __forceinline__ void fin_restart(Ctl* ctl, double rr) {
  ctl->rho = rr;
  ctl->r0norm2 = rr;
  ctl->rnorm2 = rr;
  ctl->alpha = 1.0;
  ctl->omega = 1.0;
  ctl->beta = 0.0;
  ctl->since = 0;
  ctl->fresh = 1;
  ctl->rsel = 1;
  ctl->r0sel = 1;
  ctl->state = !isfinite(rr) ? ST_NONFINITE : (rr <= ctl->stop2 ? ST_CONVERGED : ST_RUNNING);
}
// alpha = rho / <r0, v>; a zero or non-finite value is a breakdown: restart
__device__ __forceinline__ void fin_alpha(Ctl* ctl, double rv) {
  const double alpha = ctl->rho / rv;
  if (rv == 0.0 || !isfinite(alpha)) {
    ctl->iter += 1;
    ctl->restarts += 1;
    ctl->state = ctl->iter >= ctl->maxit ? ST_MAXIT : ST_RESTART;
  } else {
    ctl->alpha = alpha;
  }
}
// ||s||^2: half-step exit when it meets the tolerance
__device__ __forceinline__ void fin_snorm(Ctl* ctl, double ss) {
  ctl->snorm2 = ss;
  if (!isfinite(ss))
    ctl->state = ST_NONFINITE;
  else if (ss <= ctl->stop2)
    ctl->state = ST_HALF;
}
// omega = <t, s> / <t, t>
__device__ __forceinline__ void fin_omega(Ctl* ctl, double ts, double tt) {
  const double omega = tt > 0.0 ? ts / tt : 0.0;
  if (!isfinite(omega)) ctl->state = ST_NONFINITE;
  ctl->omega = omega;
}
// end of an iteration: stop, restart (every restart_every iterations, Sec. 4,
// or on breakdown) or beta = (rho'/rho)(alpha/omega).  Returns the new state.
__device__ __forceinline__ int fin_iteration(Ctl* ctl, bool half, double rho1, double rr) {
  int st;
  ctl->iter += 1;
  ctl->since += 1;
  ctl->xzero = 0;
  if (half) {
    ctl->rnorm2 = ctl->snorm2;
    st = ST_CONVERGED;
  } else {
    ctl->rnorm2 = rr;
    ctl->rsel = 1;
    ctl->fresh = 0;
    if (!isfinite(rr) || !isfinite(rho1)) {
      st = ST_NONFINITE;
    } else if (rr <= ctl->stop2) {
      st = ST_CONVERGED;
    } else if (ctl->iter >= ctl->maxit) {
      st = ST_MAXIT;
    } else if (ctl->omega == 0.0 || ctl->since >= ctl->restart_every ||
               fabs(rho1) <= 1e-14 * sqrt(ctl->r0norm2 * rr)) {
      st = ST_RESTART;
      ctl->restarts += 1;
    } else {
      ctl->beta = (rho1 / ctl->rho) * (ctl->alpha / ctl->omega);
      ctl->rho = rho1;
      st = ST_RUNNING;
    }
  }
  const int hi = ctl->hist_off + ctl->iter - 1;
  if (ctl->hist && hi < ctl->hist_cap) ctl->hist[hi] = ctl->bnorm2 > 0.0 ? sqrt(ctl->rnorm2 / ctl->bnorm2) : 0.0;
  ctl->state = st;
  return st;
}

// Restart of one column (rare, kept out of line): r = rhs - Ahat x, r0 = r,
// p = r, ph = T^-1 p.  Returns the column's <r, r>.  x is read-only here; x64
// (may be null) holds x in FP64 instead of w.x.
template <typename T>
__device__ __noinline__ double restart_column(const Grid& g, int64_t col, const Bands<T>& a, const Vecs<T>& w,
                                              bool xzero, const double* x64) {
  const ColNbr c = col_nbr(g, col);
  T cacc = T(0);
  for (int k = 0; k < g.nz; ++k) {
    const int64_t idx = (int64_t)k * g.ncol + col;
    T rk = w.rhs[idx];
    if (!xzero) rk -= x64 ? ahat_point(g, a, x64, idx, k, c) : ahat_point(g, a, w.x, idx, k, c);
    w.r[idx] = rk;
    w.r0[idx] = rk;
    cacc = fma(rk, rk, cacc);
  }
  // r was written just above, in this launch: coherent loads (the read-only
  // path may serve a line cached before the write)
  SrcCopy<T, 1, LD_PLAIN> src{w.r, w.p};
  thomas_vec<T, 1, 4>(g, col, a.m, a.l, a.cp, w.ph, src);
  return (double)cacc;
}

// ---------------------------------------------------------------------------
// k_pre_p: p = r + beta (p - omega v), ph = T^-1 p (the common case).
// dynamic shared memory of the variants that park the forward sweep there
extern __shared__ __align__(16) unsigned char hz_park[];

template <typename T, int V, int U, int P>
__global__ void __launch_bounds__(kBS, kMinBlocks) k_pre_p(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl) {
  if (ctl->state != ST_RUNNING || ctl->fresh) return;
  using S = SrcP<T, V, LD_NC, P == PARK_OUT_L2>;
  T* ys = reinterpret_cast<T*>(hz_park);
  const T beta = (T)ctl->beta, omega = (T)ctl->omega;
  const T* __restrict__ rin = ctl->rsel ? w.r : w.rhs;
  const int64_t ng = g.ncol / V;
  for (int64_t q = (int64_t)blockIdx.x * kBS + threadIdx.x; q < ng; q += (int64_t)gridDim.x * kBS) {
    S src{rin, w.p, w.v, beta, omega};
    thomas_vec<T, V, U, S, P>(g, q * V, a.m, a.l, a.cp, w.ph, src, ys);
  }
}

// k_pre_start: the first iteration after a start (p = r, ph = T^-1 p) or a
// restart (Sec. 4): r = rhs - Ahat x, r0 = r, ||r||^2, p = r, ph = T^-1 p.
// Launched every iteration, it returns at once in every other state, so the
// common path carries no registers for the rare one.
template <typename T>
__global__ void __launch_bounds__(kBS, 4) k_pre_start(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl, Red red) {
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->bodies += 1;  // read only by k_upd, a later launch
  const int state = ctl->state;
  const bool restart = (state == ST_RESTART);
  if (!restart && !(state == ST_RUNNING && ctl->fresh)) return;
  const bool xzero = ctl->xzero != 0;
  const bool f32 = sizeof(T) == 4 && ctl->dot32;
  const double* x64 = sizeof(T) == 4 ? ctl->x64 : nullptr;
  const T* __restrict__ rin = ctl->rsel ? w.r : w.rhs;
  double acc = 0.0;
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    if (restart) {
      acc = acc_add(acc, restart_column<T>(g, col, a, w, xzero, x64), f32);
    } else {
      SrcCopy<T, 1> src{rin, w.p};
      thomas_vec<T, 1, 8>(g, col, a.m, a.l, a.cp, w.ph, src);
    }
  }
  if (restart) {
    double vv[1] = {acc}, out[1];
    if (grid_reduce<1>(vv, red, out, f32)) fin_restart(ctl, out[0]);
  }
}

// ---------------------------------------------------------------------------
// k_mv<0>: v = p + H ph and <r0, v>  ->  alpha = rho / <r0, v>
// k_mv<1>: t = s + H sh, <t, s>, <t, t> and <s, s>  ->  the half-step exit
// test on ||s|| (it reads every s anyway, so the test costs no traffic here;
// in the Thomas sweep of k_pre_s the running sum slowed the sweep by a sixth),
// then omega = <t,s>/<t,t>
template <typename T, int MODE, int V, int U, bool H, int HB = HB_F32>
__global__ void __launch_bounds__(kBS, kMinBlocks) k_mv(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl, Red red) {
  if (ctl->state != ST_RUNNING) return;
  const T* __restrict__ cen = MODE == 0 ? w.p : w.s;
  const T* __restrict__ x = MODE == 0 ? w.ph : w.sh;
  T* __restrict__ y = MODE == 0 ? w.v : w.t;
  const T* __restrict__ r0 = ctl->r0sel ? w.r0 : w.rhs;
  const bool f32 = sizeof(T) == 4 && ctl->dot32;
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
  const int64_t ng = g.ncol / V;
  for (int64_t q = (int64_t)blockIdx.x * kBS + threadIdx.x; q < ng; q += (int64_t)gridDim.x * kBS)
    hmv_vec<T, V, U, MODE == 0 ? 0 : 3, LD_NC, H, HB>(g, q * V, a, cen, x, y, r0, acc0, acc1, &acc2, f32);
  if (MODE == 0) {
    double vv[1] = {acc0}, out[1];
    if (grid_reduce<1>(vv, red, out, f32)) fin_alpha(ctl, out[0]);
  } else {
    double vv[3] = {acc0, acc1, acc2}, out[3];
    if (grid_reduce<3>(vv, red, out, f32)) {
      fin_snorm(ctl, out[2]);
      if (ctl->state == ST_RUNNING) fin_omega(ctl, out[0], out[1]);
    }
  }
}

// ---------------------------------------------------------------------------
// k_pre_s: s = r - alpha v, sh = T^-1 s (the half-step test on ||s|| follows in k_mv<1>)
template <typename T, int V, int U, int P>
__global__ void __launch_bounds__(kBS, kMinBlocks) k_pre_s(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl) {
  if (ctl->state != ST_RUNNING) return;
  using S = SrcS<T, V, LD_NC, P == PARK_OUT_L2, false>;
  T* ys = reinterpret_cast<T*>(hz_park);
  const T alpha = (T)ctl->alpha;
  const T* __restrict__ rin = ctl->rsel ? w.r : w.rhs;
  const int64_t ng = g.ncol / V;
  for (int64_t q = (int64_t)blockIdx.x * kBS + threadIdx.x; q < ng; q += (int64_t)gridDim.x * kBS) {
    S src{rin, w.v, w.s, alpha, T(0), {}};
    thomas_vec<T, V, U, S, P>(g, q * V, a.m, a.l, a.cp, w.sh, src, ys);
  }
}

// ---------------------------------------------------------------------------
// k_upd: x += alpha ph + omega sh; r = s - omega t; <r0, r>, <r, r>; then the
// control step: stop, restart (every `restart_every` iterations, Sec. 4, or on
// breakdown) or beta = (rho'/rho)(alpha/omega).  Elementwise, vectorised.
template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
  static constexpr int W = 4;
};
template <>
struct Vec4<double> {
  using type = double2;
  static constexpr int W = 2;
};

template <typename V, typename T>
__device__ __forceinline__ void vload(const T* p, T (&o)[sizeof(V) / sizeof(T)]) {
  V t = *reinterpret_cast<const V*>(p);
  const T* q = reinterpret_cast<const T*>(&t);
#pragma unroll
  for (int u = 0; u < (int)(sizeof(V) / sizeof(T)); ++u) o[u] = q[u];
}
template <typename V, typename T>
__device__ __forceinline__ void vstore(T* p, const T (&o)[sizeof(V) / sizeof(T)]) {
  V t;
  T* q = reinterpret_cast<T*>(&t);
#pragma unroll
  for (int u = 0; u < (int)(sizeof(V) / sizeof(T)); ++u) q[u] = o[u];
  *reinterpret_cast<V*>(p) = t;
}

template <typename T>
__global__ void __launch_bounds__(256) k_upd(Grid g, Vecs<T> w, Ctl* ctl, Red red, cudaGraphConditionalHandle cond,
                                              int use_cond) {
  const int state = ctl->state;
  if (ctl->bodies > ctl->body_limit) {  // hard stop of the device loop (the host reports MAXIT)
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  if (state != ST_RUNNING && state != ST_HALF) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, state == ST_RESTART ? 1u : 0u);
    return;
  }
  const bool half = (state == ST_HALF);
  const bool xzero = ctl->xzero != 0;
  const bool f32 = sizeof(T) == 4 && ctl->dot32;
  // the paper's mixed-precision solver keeps x in FP64 (updated in FP64 from
  // the FP32 vectors and the FP64 scalars); otherwise x is a T vector
  double* __restrict__ x64 = sizeof(T) == 4 ? ctl->x64 : nullptr;
  const double alpha_d = ctl->alpha, omega_d = ctl->omega;
  const T alpha = (T)alpha_d, omega = (T)omega_d;
  const T* __restrict__ r0 = ctl->r0sel ? w.r0 : w.rhs;
  T* __restrict__ x = w.x;
  T* __restrict__ r = w.r;
  const T* __restrict__ ph = w.ph;
  const T* __restrict__ sh = w.sh;
  const T* __restrict__ s = w.s;
  const T* __restrict__ t = w.t;
  using V = typename Vec4<T>::type;
  constexpr int VW = Vec4<T>::W;
  DotAcc<T> acc0{}, acc1{};
  const int64_t n = g.n;
  const int64_t nv = (n % VW == 0) ? n / VW : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += stride) {
    const int64_t e = q * VW;
    T xv[VW], pv[VW], shv[VW];
    if (!x64) {  // loads in the order of the streams: x, ph, then sh, s, t, r0
      if (xzero) {
#pragma unroll
        for (int u = 0; u < VW; ++u) xv[u] = T(0);
      } else {
        vload<V>(x + e, xv);
      }
    }
    vload<V>(ph + e, pv);
    if (!half) {
      T sv[VW], tv[VW], r0v[VW], rv[VW];
      vload<V>(sh + e, shv);
      vload<V>(s + e, sv);
      vload<V>(t + e, tv);
      vload<V>(r0 + e, r0v);
      T a0 = T(0), a1 = T(0);
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        rv[u] = fma(-omega, tv[u], sv[u]);
        a0 = fma(r0v[u], rv[u], a0);
        a1 = fma(rv[u], rv[u], a1);
      }
      vstore<V>(r + e, rv);
      acc0.add(a0);
      acc1.add(a1);
    }
    if (x64) {
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        double xd = xzero ? 0.0 : x64[e + u];
        xd = fma(alpha_d, (double)pv[u], xd);
        if (!half) xd = fma(omega_d, (double)shv[u], xd);
        x64[e + u] = xd;
      }
      continue;
    }
    if (half) {
#pragma unroll
      for (int u = 0; u < VW; ++u) xv[u] = fma(alpha, pv[u], xv[u]);
    } else {
#pragma unroll
      for (int u = 0; u < VW; ++u) xv[u] = fma(omega, shv[u], fma(alpha, pv[u], xv[u]));
    }
    vstore<V>(x + e, xv);
  }
  if (nv == 0) {  // scalar path for sizes that are not a multiple of the vector width
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
      if (x64) {
        double xd = xzero ? 0.0 : x64[e];
        xd = fma(alpha_d, (double)ph[e], xd);
        if (!half) xd = fma(omega_d, (double)sh[e], xd);
        x64[e] = xd;
      } else {
        T xv = xzero ? T(0) : x[e];
        xv = fma(alpha, ph[e], xv);
        if (!half) xv = fma(omega, sh[e], xv);
        x[e] = xv;
      }
      if (!half) {
        const T rv = fma(-omega, t[e], s[e]);
        r[e] = rv;
        acc0.add(r0[e] * rv);
        acc1.add(rv * rv);
      }
    }
  }
  double vv[2] = {acc0.total(f32), acc1.total(f32)}, out[2];
  if (grid_reduce<2>(vv, red, out, f32)) {
    const int st = fin_iteration(ctl, half, out[0], out[1]);
    if (use_cond) cudaGraphSetConditional(cond, (st == ST_RUNNING || st == ST_RESTART) ? 1u : 0u);
  }
}


// ---------------------------------------------------------------------------
// building blocks exposed for testing: the same column code as the solver
template <typename T>
__global__ void __launch_bounds__(kBS) k_matvec_hat(Grid g, Bands<T> a, const T* __restrict__ x, T* __restrict__ y) {
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    const ColNbr c = col_nbr(g, col);
    for (int k = 0; k < g.nz; ++k) {
      const int64_t idx = (int64_t)k * g.ncol + col;
      y[idx] = ahat_point(g, a, x, idx, k, c);
    }
  }
}

template <typename T, int V, int U, int P>
__global__ void __launch_bounds__(kBS, kMinBlocks) k_tinv(Grid g, Bands<T> a, const T* __restrict__ r,
                                                          T* __restrict__ z) {
  using S = SrcCopy<T, V, LD_NC, P == PARK_OUT_L2>;
  T* ys = reinterpret_cast<T*>(hz_park);
  const int64_t ng = g.ncol / V;
  for (int64_t q = (int64_t)blockIdx.x * kBS + threadIdx.x; q < ng; q += (int64_t)gridDim.x * kBS) {
    S src{r, nullptr};
    thomas_vec<T, V, U, S, P>(g, q * V, a.m, a.l, a.cp, z, src, ys);
  }
}

template <typename T, int V, int U, bool H, int HB = HB_F32>
__global__ void __launch_bounds__(kBS, kMinBlocks) k_hmv(Grid g, Bands<T> a, const T* __restrict__ cen,
                                                         const T* __restrict__ x, T* __restrict__ y) {
  const int64_t ng = g.ncol / V;
  double d0 = 0.0, d1 = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * kBS + threadIdx.x; q < ng; q += (int64_t)gridDim.x * kBS)
    hmv_vec<T, V, U, 2, LD_NC, H, HB>(g, q * V, a, cen, x, y, nullptr, d0, d1);
}

// ---- variant dispatch ----------------------------------------------------------
template <typename T, int I = 0, typename F>
cudaError_t with_pre(int var, F&& f) {
  if constexpr (I < Variants<T>::NPRE) {
    if (var == I)
      return f(std::integral_constant<int, Variants<T>::pre_v[I]>{}, std::integral_constant<int, Variants<T>::pre_u[I]>{},
               std::integral_constant<int, Variants<T>::pre_p[I]>{}, Variants<T>::pre_b[I]);
    return with_pre<T, I + 1>(var, f);
  } else {
    return cudaErrorInvalidValue;
  }
}
template <typename T, int I = 0, typename F>
cudaError_t with_mv(int var, F&& f) {
  if constexpr (I < Variants<T>::NMV) {
    if (var == I)
      return f(std::integral_constant<int, Variants<T>::mv_v[I]>{}, std::integral_constant<int, Variants<T>::mv_u[I]>{},
               std::integral_constant<bool, Variants<T>::mv_h[I] != 0>{}, Variants<T>::mv_b[I]);
    return with_mv<T, I + 1>(var, f);
  } else {
    return cudaErrorInvalidValue;
  }
}
template <typename T>
constexpr int prec_index() {
  return sizeof(T) == 8 ? 1 : 0;
}
// the band format of a launch as a compile-time value (FP64 kernels: FP64 bands)
template <typename T, typename F>
cudaError_t with_hb(int hb, F&& f) {
  if constexpr (sizeof(T) == 4) {
    if (hb == HB_BF16) return f(std::integral_constant<int, HB_BF16>{});
    if (hb == HB_FP16) return f(std::integral_constant<int, HB_FP16>{});
  }
  return f(std::integral_constant<int, HB_F32>{});
}
inline int64_t blocks_for(int64_t items, int block) { return (items + block - 1) / block; }

template <typename T>
cudaError_t launch_pre_p_t(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L) {
  k_pre_start<T><<<grid_for((const void*)k_pre_start<T>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, ctl, red);
  return with_pre<T>(L.vpre[prec_index<T>()], [&](auto Vc, auto Uc, auto Pc, int cap) {
    constexpr int V = decltype(Vc)::value, U = decltype(Uc)::value, P = decltype(Pc)::value;
    if constexpr (P == PARK_BULK) {
      if constexpr (sizeof(T) == 4) return launch_thomas_bulk(0, U, cap, g, a, w, nullptr, nullptr, ctl, &ctl->kerr, L);
      return cudaErrorInvalidValue;
    } else {
    const void* k = (const void*)k_pre_p<T, V, U, P>;
    const size_t sm = park_bytes<T, V, P>(g.nz);
    k_pre_p<T, V, U, P><<<grid_for(k, kBS, L, blocks_for(g.ncol / V, kBS), sm, cap), kBS, sm, L.stream>>>(g, a, w,
                                                                                                          ctl);
    return cudaGetLastError();
    }
  });
}
template <typename T>
cudaError_t launch_pre_s_t(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L) {
  return with_pre<T>(L.vpre[prec_index<T>()], [&](auto Vc, auto Uc, auto Pc, int cap) {
    constexpr int V = decltype(Vc)::value, U = decltype(Uc)::value, P = decltype(Pc)::value;
    if constexpr (P == PARK_BULK) {
      if constexpr (sizeof(T) == 4) return launch_thomas_bulk(1, U, cap, g, a, w, nullptr, nullptr, ctl, &ctl->kerr, L);
      return cudaErrorInvalidValue;
    } else {
    const void* k = (const void*)k_pre_s<T, V, U, P>;
    const size_t sm = park_bytes<T, V, P>(g.nz);
    k_pre_s<T, V, U, P><<<grid_for(k, kBS, L, blocks_for(g.ncol / V, kBS), sm, cap), kBS, sm, L.stream>>>(g, a, w,
                                                                                                          ctl);
    return cudaGetLastError();
    }
  });
}
template <typename T, int MODE>
cudaError_t launch_mv_t_(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L) {
  return with_mv<T>(L.vmv[prec_index<T>()], [&](auto Vc, auto Uc, auto Hc, int cap) {
    return with_hb<T>(a.h16fmt, [&](auto Bc) {
      constexpr int V = decltype(Vc)::value, U = decltype(Uc)::value, HB = decltype(Bc)::value;
      constexpr bool H = decltype(Hc)::value;
      const void* k = (const void*)k_mv<T, MODE, V, U, H, HB>;
      k_mv<T, MODE, V, U, H, HB><<<grid_for(k, kBS, L, blocks_for(g.ncol / V, kBS), 0, cap), kBS, 0, L.stream>>>(g, a, w, ctl,
                                                                                                          red);
      return cudaGetLastError();
    });
  });
}
template <typename T>
cudaError_t launch_upd_t(const Grid& g, const Vecs<T>& w, Ctl* ctl, Red red, unsigned long long cond, int use_cond,
                         const Launch& L) {
  k_upd<T><<<grid_for((const void*)k_upd<T>, 256, L, L.wflat), 256, 0, L.stream>>>(g, w, ctl, red,
                                                                                    (cudaGraphConditionalHandle)cond,
                                                                                    use_cond);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_matvec_hat_t(const Grid& g, const Bands<T>& a, const T* x, T* y, const Launch& L) {
  k_matvec_hat<T><<<grid_for((const void*)k_matvec_hat<T>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, x, y);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_tinv_t(const Grid& g, const Bands<T>& a, const T* r, T* z, const Launch& L) {
  return with_pre<T>(L.vpre[prec_index<T>()], [&](auto Vc, auto Uc, auto Pc, int cap) {
    constexpr int V = decltype(Vc)::value, U = decltype(Uc)::value, P = decltype(Pc)::value;
    if constexpr (P == PARK_BULK) {
      if constexpr (sizeof(T) == 4) return launch_thomas_bulk(2, U, cap, g, a, Vecs<T>{}, r, z, nullptr, L.err, L);
      return cudaErrorInvalidValue;
    } else {
    const void* k = (const void*)k_tinv<T, V, U, P>;
    const size_t sm = park_bytes<T, V, P>(g.nz);
    k_tinv<T, V, U, P><<<grid_for(k, kBS, L, blocks_for(g.ncol / V, kBS), sm, cap), kBS, sm, L.stream>>>(g, a, r, z);
    return cudaGetLastError();
    }
  });
}
template <typename T>
cudaError_t launch_precond_matvec_t(const Grid& g, const Bands<T>& a, const T* p, T* ph, T* v, const Launch& L) {
  cudaError_t e = launch_tinv_t<T>(g, a, p, ph, L);
  if (e != cudaSuccess) return e;
  return with_mv<T>(L.vmv[prec_index<T>()], [&](auto Vc, auto Uc, auto Hc, int cap) {
    return with_hb<T>(a.h16fmt, [&](auto Bc) {
      constexpr int V = decltype(Vc)::value, U = decltype(Uc)::value, HB = decltype(Bc)::value;
      constexpr bool H = decltype(Hc)::value;
      const void* k = (const void*)k_hmv<T, V, U, H, HB>;
      k_hmv<T, V, U, H, HB><<<grid_for(k, kBS, L, blocks_for(g.ncol / V, kBS), 0, cap), kBS, 0, L.stream>>>(g, a, p, ph, v);
      return cudaGetLastError();
    });
  });
}

// query the occupancy of every kernel of precision T once, outside any capture
template <typename T>
void warm_t(const Launch& L) {
  grid_for((const void*)k_pre_start<T>, kBS, L, 1);
  grid_for((const void*)k_upd<T>, 256, L, 1);
  grid_for((const void*)k_matvec_hat<T>, kBS, L, 1);
  for (int i = 0; i < Variants<T>::NPRE; ++i)
    with_pre<T>(i, [&](auto Vc, auto Uc, auto Pc, int) {
      constexpr int V = decltype(Vc)::value, U = decltype(Uc)::value, P = decltype(Pc)::value;
      if constexpr (P == PARK_BULK) {
        if (sizeof(T) == 4) warm_thomas_bulk(L, L.nz);
        return cudaSuccess;
      } else {
        constexpr bool SM = P == PARK_SMEM;
        const size_t sm = park_bytes<T, V, P>(L.nz);
        const void* ks[3] = {(const void*)k_pre_p<T, V, U, P>, (const void*)k_pre_s<T, V, U, P>,
                             (const void*)k_tinv<T, V, U, P>};
        for (const void* k : ks) {
          if (sm > kParkMax) continue;  // the variant is not valid for this nz
          if (SM &&
              cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kParkMax) != cudaSuccess)
            cudaGetLastError();  // the launch reports it; nothing stale is left behind
          grid_for(k, kBS, L, 1, sm);
        }
        return cudaSuccess;
      }
    });
  for (int i = 0; i < Variants<T>::NMV; ++i)
    for (int hb = HB_F32; hb <= (sizeof(T) == 4 ? HB_FP16 : HB_F32); ++hb)
      with_mv<T>(i, [&](auto Vc, auto Uc, auto Hc, int) {
        return with_hb<T>(hb, [&](auto Bc) {
          constexpr int V = decltype(Vc)::value, U = decltype(Uc)::value, HB = decltype(Bc)::value;
          constexpr bool H = decltype(Hc)::value;
          grid_for((const void*)k_mv<T, 0, V, U, H, HB>, kBS, L, 1);
          grid_for((const void*)k_mv<T, 1, V, U, H, HB>, kBS, L, 1);
          grid_for((const void*)k_hmv<T, V, U, H, HB>, kBS, L, 1);
          return cudaSuccess;
        });
      });
}

}  // namespace hz
