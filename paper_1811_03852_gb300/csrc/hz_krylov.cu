// hz_krylov.cu -- the inner BiCGStab iteration on sm_103a.
//
// Right-preconditioned ("post-conditioned", Maynard & Walters Sec. 2)
// BiCGStab (van der Vorst 1992) on Ahat y = rhs with C = T^-1.  One iteration
// is five launches; every scalar lives in the device control block, so the
// loop needs no host round trip and can run as a CUDA-graph while loop:
//
//   k_pre_p : p = r + beta (p - omega v)           then ph = T^-1 p     (Thomas, column per thread)
//   k_mv<0> : v = p + H ph,  <r0, v>  -> alpha     (T ph = p, so Ahat ph = p + H ph)
//   k_pre_s : s = r - alpha v, <s, s>              then sh = T^-1 s
//   k_mv<1> : t = s + H sh,  <t, s>, <t, t> -> omega
//   k_upd   : x += alpha ph + omega sh, r = s - omega t, <r0, r>, <r, r> -> beta, stop/restart
//
// H = the four horizontal bands (E, W, N, S) of Ahat.  Layout [k][j][i]: a
// thread owns one column (i, j) and marches k, so every load of a warp is a
// contiguous 128-byte (FP32) or 256-byte (FP64) run.  The k-march is
// software-pipelined: the loads of U consecutive levels are issued together
// before any of them is used, which keeps enough bytes in flight per SM for
// HBM while the Thomas recurrence stays sequential in k.  Partial sums are
// FP32 (FP64 in the FP64 solver) over one column and FP64 across threads and
// blocks (the paper's 64-bit global sums, Sec. 4); the grid reduction is
// deterministic (fixed slots, summed in slot order by the last block).
#include <mutex>
#include <unordered_map>
#include <vector>

#include "hz_internal.cuh"

namespace hz {

// levels per software-pipelined batch: Thomas sweeps and the stencil
template <typename T>
struct Tune;
template <>
struct Tune<float> {
  static constexpr int UT = 8, UM = 4, MINB = 6;
};
template <>
struct Tune<double> {
  static constexpr int UT = 4, UM = 2, MINB = 6;
};

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

// (Ahat x)_idx with all six bands (used on restart and by the test entry point)
template <typename T>
__device__ __forceinline__ T ahat_point(const Grid& g, const Bands<T>& a, const T* __restrict__ x, int64_t idx, int k,
                                        const ColNbr& c) {
  T y = x[idx];
  y = fma(a.E[idx], x[idx + c.ie], y);
  y = fma(a.W[idx], x[idx + c.iw], y);
  if (c.hn) y = fma(a.N[idx], x[idx + g.nx], y);
  if (c.hs) y = fma(a.S[idx], x[idx - g.nx], y);
  if (k + 1 < g.nz) y = fma(a.U[idx], x[idx + g.ncol], y);
  if (k > 0) y = fma(a.D[idx], x[idx - g.ncol], y);
  return y;
}

// Thomas algorithm on one column with unit diagonal and pre-computed factors:
// forward y_k = m_k q_k - l_k y_(k-1), back z_k = y_k - c'_k z_(k+1).  The
// input q_k comes from src.make(v, idx) on the src.NIN values that src.load
// fetched for level k (the fused axpy).  y is parked in out and re-read by the
// back sweep (an L2 hit: the whole resident wave's columns fit in L2).
template <typename T, int U, typename Src>
__device__ __forceinline__ void thomas_batched(const Grid& g, int64_t col, const T* __restrict__ m,
                                               const T* __restrict__ l, const T* __restrict__ cp,
                                               T* __restrict__ out, Src& src) {
  constexpr int NIN = Src::NIN;
  const int64_t ncol = g.ncol;
  const int nz = g.nz;
  T yprev = T(0);
  for (int k0 = 0; k0 < nz; k0 += U) {
    T v[U][NIN], mm[U], ll[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + col;
        src.load(idx, v[u]);
        mm[u] = ldro(m + idx);
        ll[u] = ldro(l + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + col;
        const T q = src.make(v[u], idx);
        const T y = fma(mm[u], q, -ll[u] * yprev);
        out[idx] = y;
        yprev = y;
      }
    }
  }
  T zn = T(0);
  for (int k0 = nz - 1; k0 >= 0; k0 -= U) {
    T yy[U], cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 - u >= 0) {
        const int64_t idx = (int64_t)(k0 - u) * ncol + col;
        yy[u] = out[idx];  // written by this thread above: coherent load
        cc[u] = ldro(cp + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 - u >= 0) {
        const int64_t idx = (int64_t)(k0 - u) * ncol + col;
        const T z = fma(-cc[u], zn, yy[u]);
        out[idx] = z;
        zn = z;
      }
    }
  }
}

// inputs of the Thomas sweeps
template <typename T>
struct SrcP {  // p = r + beta (p - omega v)
  static constexpr int NIN = 3;
  const T* __restrict__ r;
  T* __restrict__ p;
  const T* __restrict__ v;
  T beta, omega;
  __device__ __forceinline__ void load(int64_t idx, T (&o)[NIN]) {
    o[0] = ldro(r + idx);
    o[1] = p[idx];
    o[2] = ldro(v + idx);
  }
  __device__ __forceinline__ T make(const T (&o)[NIN], int64_t idx) {
    const T pk = fma(beta, fma(-omega, o[2], o[1]), o[0]);
    p[idx] = pk;
    return pk;
  }
};

template <typename T>
struct SrcCopy {  // p = r (first iteration after a start); dst may be null
  static constexpr int NIN = 1;
  const T* __restrict__ r;
  T* __restrict__ dst;
  __device__ __forceinline__ void load(int64_t idx, T (&o)[NIN]) { o[0] = ldro(r + idx); }
  __device__ __forceinline__ T make(const T (&o)[NIN], int64_t idx) {
    if (dst) dst[idx] = o[0];
    return o[0];
  }
};

template <typename T>
struct SrcS {  // s = r - alpha v, accumulating <s, s>
  static constexpr int NIN = 2;
  const T* __restrict__ r;
  const T* __restrict__ v;
  T* __restrict__ s;
  T alpha;
  T acc;
  __device__ __forceinline__ void load(int64_t idx, T (&o)[NIN]) {
    o[0] = ldro(r + idx);
    o[1] = ldro(v + idx);
  }
  __device__ __forceinline__ T make(const T (&o)[NIN], int64_t idx) {
    const T sk = fma(-alpha, o[1], o[0]);
    s[idx] = sk;
    acc = fma(sk, sk, acc);
    return sk;
  }
};

// Restart of one column (rare, kept out of line so that it does not cost the
// common path registers): r = rhs - Ahat x, r0 = r, p = r, ph = T^-1 p.
// Returns the column's <r, r>.  x is read-only in this launch.
template <typename T>
__device__ __noinline__ double restart_column(const Grid& g, int64_t col, const Bands<T>& a, const Vecs<T>& w,
                                              bool xzero) {
  const ColNbr c = col_nbr(g, col);
  T cacc = T(0);
  for (int k = 0; k < g.nz; ++k) {
    const int64_t idx = (int64_t)k * g.ncol + col;
    T rk = w.rhs[idx];
    if (!xzero) rk -= ahat_point(g, a, w.x, idx, k, c);
    w.r[idx] = rk;
    w.r0[idx] = rk;
    cacc = fma(rk, rk, cacc);
  }
  SrcCopy<T> src{w.r, w.p};
  thomas_batched<T, Tune<T>::UT>(g, col, a.m, a.l, a.cp, w.ph, src);
  return (double)cacc;
}

// ---------------------------------------------------------------------------
// k_pre_p: p = r + beta (p - omega v), ph = T^-1 p (the common case).
// k_pre_start does the first iteration after a start (p = r) and the restart
// (Sec. 4: the mandatory restart): r = rhs - Ahat x, r0 = r, ||r||^2, p = r.
// Both are launched every iteration; each returns at once when the state is
// not its own, so the common path carries no registers for the rare one.
template <typename T>
__global__ void __launch_bounds__(kBS, Tune<T>::MINB) k_pre_p(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl) {
  if (ctl->state != ST_RUNNING || ctl->fresh) return;
  const T beta = (T)ctl->beta, omega = (T)ctl->omega;
  const T* __restrict__ rin = ctl->rsel ? w.r : w.rhs;
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    SrcP<T> src{rin, w.p, w.v, beta, omega};
    thomas_batched<T, Tune<T>::UT>(g, col, a.m, a.l, a.cp, w.ph, src);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBS, 4) k_pre_start(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl, Red red) {
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->bodies += 1;  // read only by k_upd, a later launch
  const int state = ctl->state;
  const bool restart = (state == ST_RESTART);
  if (!restart && !(state == ST_RUNNING && ctl->fresh)) return;
  const bool xzero = ctl->xzero != 0;
  const T* __restrict__ rin = ctl->rsel ? w.r : w.rhs;
  double acc = 0.0;
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    if (restart) {
      acc += restart_column<T>(g, col, a, w, xzero);
    } else {
      SrcCopy<T> src{rin, w.p};
      thomas_batched<T, Tune<T>::UT>(g, col, a.m, a.l, a.cp, w.ph, src);
    }
  }
  if (restart) {
    double vv[1] = {acc}, out[1];
    if (grid_reduce<1>(vv, red, out)) {
      const double rr = out[0];
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
  }
}

// ---------------------------------------------------------------------------
// y = c + H x over one column, U levels per batch; a0/a1 accumulate the dots.
// MODE 0: a0 += r0 y.  MODE 1: a0 += y c, a1 += y y.
template <typename T, int U, int MODE>
__device__ __forceinline__ void hmv_column(const Grid& g, int64_t col, const Bands<T>& a, const T* __restrict__ cen,
                                           const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ r0,
                                           T& a0, T& a1) {
  const ColNbr c = col_nbr(g, col);
  const int64_t ncol = g.ncol, nx = g.nx;
  for (int k0 = 0; k0 < g.nz; k0 += U) {
    T cc[U], e[U], w[U], nn[U], ss[U], xe[U], xw[U], xn[U], xs[U], q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < g.nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + col;
        cc[u] = ldro(cen + idx);
        e[u] = ldro(a.E + idx);
        w[u] = ldro(a.W + idx);
        xe[u] = ldro(x + idx + c.ie);
        xw[u] = ldro(x + idx + c.iw);
        nn[u] = c.hn ? ldro(a.N + idx) : T(0);
        xn[u] = c.hn ? ldro(x + idx + nx) : T(0);
        ss[u] = c.hs ? ldro(a.S + idx) : T(0);
        xs[u] = c.hs ? ldro(x + idx - nx) : T(0);
        if (MODE == 0) q[u] = ldro(r0 + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < g.nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + col;
        T yy = fma(e[u], xe[u], cc[u]);
        yy = fma(w[u], xw[u], yy);
        yy = fma(nn[u], xn[u], yy);
        yy = fma(ss[u], xs[u], yy);
        y[idx] = yy;
        if (MODE == 0) {
          a0 = fma(q[u], yy, a0);
        } else {
          a0 = fma(yy, cc[u], a0);
          a1 = fma(yy, yy, a1);
        }
      }
    }
  }
}

// k_mv<0>: v = p + H ph and <r0, v>  ->  alpha = rho / <r0, v>
// k_mv<1>: t = s + H sh, <t, s> and <t, t>  ->  omega = <t,s>/<t,t>
template <typename T, int MODE>
__global__ void __launch_bounds__(kBS, Tune<T>::MINB) k_mv(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl, Red red) {
  if (ctl->state != ST_RUNNING) return;
  const T* __restrict__ cen = MODE == 0 ? w.p : w.s;
  const T* __restrict__ x = MODE == 0 ? w.ph : w.sh;
  T* __restrict__ y = MODE == 0 ? w.v : w.t;
  const T* __restrict__ r0 = ctl->r0sel ? w.r0 : w.rhs;
  double acc0 = 0.0, acc1 = 0.0;
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    T a0 = T(0), a1 = T(0);
    hmv_column<T, Tune<T>::UM, MODE>(g, col, a, cen, x, y, r0, a0, a1);
    acc0 += (double)a0;
    acc1 += (double)a1;
  }
  if (MODE == 0) {
    double vv[1] = {acc0}, out[1];
    if (grid_reduce<1>(vv, red, out)) {
      const double rv = out[0];
      const double alpha = ctl->rho / rv;
      if (rv == 0.0 || !isfinite(alpha)) {
        // breakdown of the Lanczos part: count the iteration and restart
        ctl->iter += 1;
        ctl->restarts += 1;
        ctl->state = ctl->iter >= ctl->maxit ? ST_MAXIT : ST_RESTART;
      } else {
        ctl->alpha = alpha;
      }
    }
  } else {
    double vv[2] = {acc0, acc1}, out[2];
    if (grid_reduce<2>(vv, red, out)) {
      const double ts = out[0], tt = out[1];
      const double omega = tt > 0.0 ? ts / tt : 0.0;
      if (!isfinite(omega)) ctl->state = ST_NONFINITE;
      ctl->omega = omega;
    }
  }
}

// ---------------------------------------------------------------------------
// k_pre_s: s = r - alpha v, <s, s> (half-step exit test), sh = T^-1 s
template <typename T>
__global__ void __launch_bounds__(kBS, Tune<T>::MINB) k_pre_s(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl, Red red) {
  if (ctl->state != ST_RUNNING) return;
  const T alpha = (T)ctl->alpha;
  const T* __restrict__ rin = ctl->rsel ? w.r : w.rhs;
  double acc = 0.0;
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    SrcS<T> src{rin, w.v, w.s, alpha, T(0)};
    thomas_batched<T, Tune<T>::UT>(g, col, a.m, a.l, a.cp, w.sh, src);
    acc += (double)src.acc;
  }
  double vv[1] = {acc}, out[1];
  if (grid_reduce<1>(vv, red, out)) {
    const double ss = out[0];
    ctl->snorm2 = ss;
    if (!isfinite(ss))
      ctl->state = ST_NONFINITE;
    else if (ss <= ctl->stop2)
      ctl->state = ST_HALF;
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
  const T alpha = (T)ctl->alpha, omega = (T)ctl->omega;
  const T* __restrict__ r0 = ctl->r0sel ? w.r0 : w.rhs;
  T* __restrict__ x = w.x;
  T* __restrict__ r = w.r;
  const T* __restrict__ ph = w.ph;
  const T* __restrict__ sh = w.sh;
  const T* __restrict__ s = w.s;
  const T* __restrict__ t = w.t;
  using V = typename Vec4<T>::type;
  constexpr int VW = Vec4<T>::W;
  double acc0 = 0.0, acc1 = 0.0;
  const int64_t n = g.n;
  const int64_t nv = (n % VW == 0) ? n / VW : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += stride) {
    const int64_t e = q * VW;
    T xv[VW], pv[VW];
    if (xzero) {
#pragma unroll
      for (int u = 0; u < VW; ++u) xv[u] = T(0);
    } else {
      vload<V>(x + e, xv);
    }
    vload<V>(ph + e, pv);
    if (half) {
#pragma unroll
      for (int u = 0; u < VW; ++u) xv[u] = fma(alpha, pv[u], xv[u]);
      vstore<V>(x + e, xv);
    } else {
      T shv[VW], sv[VW], tv[VW], r0v[VW], rv[VW];
      vload<V>(sh + e, shv);
      vload<V>(s + e, sv);
      vload<V>(t + e, tv);
      vload<V>(r0 + e, r0v);
      T a0 = T(0), a1 = T(0);
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        xv[u] = fma(omega, shv[u], fma(alpha, pv[u], xv[u]));
        rv[u] = fma(-omega, tv[u], sv[u]);
        a0 = fma(r0v[u], rv[u], a0);
        a1 = fma(rv[u], rv[u], a1);
      }
      vstore<V>(x + e, xv);
      vstore<V>(r + e, rv);
      acc0 += (double)a0;
      acc1 += (double)a1;
    }
  }
  if (nv == 0) {  // scalar path for sizes that are not a multiple of the vector width
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
      T xv = xzero ? T(0) : x[e];
      xv = fma(alpha, ph[e], xv);
      if (!half) {
        xv = fma(omega, sh[e], xv);
        const T rv = fma(-omega, t[e], s[e]);
        r[e] = rv;
        acc0 += (double)(r0[e] * rv);
        acc1 += (double)(rv * rv);
      }
      x[e] = xv;
    }
  }
  double vv[2] = {acc0, acc1}, out[2];
  if (grid_reduce<2>(vv, red, out)) {
    int st;
    ctl->iter += 1;
    ctl->since += 1;
    ctl->xzero = 0;
    if (half) {
      ctl->rnorm2 = ctl->snorm2;
      st = ST_CONVERGED;
    } else {
      const double rho1 = out[0], rr = out[1];
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
    if (use_cond) cudaGraphSetConditional(cond, (st == ST_RUNNING || st == ST_RESTART) ? 1u : 0u);
  }
}

// ---------------------------------------------------------------------------
// building blocks exposed for testing
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

template <typename T>
__global__ void __launch_bounds__(kBS) k_tinv(Grid g, Bands<T> a, const T* __restrict__ r, T* __restrict__ z) {
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    SrcCopy<T> src{r, nullptr};
    thomas_batched<T, Tune<T>::UT>(g, col, a.m, a.l, a.cp, z, src);
  }
}

// y = c + H x with the solver's stencil code
template <typename T>
__global__ void __launch_bounds__(kBS) k_hmv(Grid g, Bands<T> a, const T* __restrict__ cen, const T* __restrict__ x,
                                             T* __restrict__ y) {
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    T a0 = T(0), a1 = T(0);
    hmv_column<T, Tune<T>::UM, 1>(g, col, a, cen, x, y, nullptr, a0, a1);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_dot(int64_t n, const T* __restrict__ x, const T* __restrict__ y, Red red,
                                             double* out_dev) {
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    acc += (double)x[e] * (double)y[e];
  double vv[1] = {acc}, out[1];
  if (grid_reduce<1>(vv, red, out)) *out_dev = out[0];
}

// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_pre_p(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L) {
  k_pre_start<T><<<grid_for((const void*)k_pre_start<T>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, ctl, red);
  k_pre_p<T><<<grid_for((const void*)k_pre_p<T>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, ctl);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_mv_v(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L) {
  k_mv<T, 0><<<grid_for((const void*)k_mv<T, 0>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, ctl, red);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_pre_s(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L) {
  k_pre_s<T><<<grid_for((const void*)k_pre_s<T>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, ctl, red);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_mv_t(const Grid& g, const Bands<T>& a, const Vecs<T>& w, Ctl* ctl, Red red, const Launch& L) {
  k_mv<T, 1><<<grid_for((const void*)k_mv<T, 1>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, ctl, red);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_upd(const Grid& g, const Vecs<T>& w, Ctl* ctl, Red red, unsigned long long cond, int use_cond,
                       const Launch& L) {
  k_upd<T><<<grid_for((const void*)k_upd<T>, 256, L, L.wflat), 256, 0, L.stream>>>(g, w, ctl, red, (cudaGraphConditionalHandle)cond, use_cond);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_matvec_hat(const Grid& g, const Bands<T>& a, const T* x, T* y, const Launch& L) {
  k_matvec_hat<T><<<grid_for((const void*)k_matvec_hat<T>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, x, y);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_tinv(const Grid& g, const Bands<T>& a, const T* r, T* z, const Launch& L) {
  k_tinv<T><<<grid_for((const void*)k_tinv<T>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, r, z);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_precond_matvec(const Grid& g, const Bands<T>& a, const T* p, T* ph, T* v, const Launch& L) {
  k_tinv<T><<<grid_for((const void*)k_tinv<T>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, p, ph);
  k_hmv<T><<<grid_for((const void*)k_hmv<T>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, p, ph, v);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_dot(int64_t n, const T* x, const T* y, Red red, double* out_dev, int grid, cudaStream_t s) {
  k_dot<T><<<grid, 256, 0, s>>>(n, x, y, red, out_dev);
  return cudaGetLastError();
}

#define HZ_INST(T)                                                                                               \
  template cudaError_t launch_pre_p<T>(const Grid&, const Bands<T>&, const Vecs<T>&, Ctl*, Red, const Launch&); \
  template cudaError_t launch_mv_v<T>(const Grid&, const Bands<T>&, const Vecs<T>&, Ctl*, Red, const Launch&);  \
  template cudaError_t launch_pre_s<T>(const Grid&, const Bands<T>&, const Vecs<T>&, Ctl*, Red, const Launch&); \
  template cudaError_t launch_mv_t<T>(const Grid&, const Bands<T>&, const Vecs<T>&, Ctl*, Red, const Launch&);  \
  template cudaError_t launch_upd<T>(const Grid&, const Vecs<T>&, Ctl*, Red, unsigned long long, int,           \
                                     const Launch&);                                                             \
  template cudaError_t launch_matvec_hat<T>(const Grid&, const Bands<T>&, const T*, T*, const Launch&);          \
  template cudaError_t launch_tinv<T>(const Grid&, const Bands<T>&, const T*, T*, const Launch&);                \
  template cudaError_t launch_precond_matvec<T>(const Grid&, const Bands<T>&, const T*, T*, T*, const Launch&);  \
  template cudaError_t launch_dot<T>(int64_t, const T*, const T*, Red, double*, int, cudaStream_t);

HZ_INST(float)
HZ_INST(double)

namespace {
std::mutex g_occ_mu;
std::unordered_map<const void*, int> g_occ;  // blocks per SM of each kernel at its block size
}  // namespace

int grid_for(const void* kernel, int block, const Launch& L, int64_t work_blocks) {
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ.find(kernel);
    if (it != g_occ.end()) {
      per_sm = it->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      g_occ[kernel] = per_sm;
    }
  }
  int64_t gsz = (int64_t)per_sm * L.sms;
  if (gsz > work_blocks) gsz = work_blocks;
  if (gsz > kMaxGrid) gsz = kMaxGrid;
  return gsz < 1 ? 1 : (int)gsz;
}

void warm_launch_kernels(const Launch& L);  // hz_setup.cu

void warm_launch_cache(const Launch& L) {
#define HZ_WARM(T)                                                       \
  grid_for((const void*)k_pre_start<T>, kBS, L, 1);                      \
  grid_for((const void*)k_pre_p<T>, kBS, L, 1);                          \
  grid_for((const void*)k_mv<T, 0>, kBS, L, 1);                          \
  grid_for((const void*)k_mv<T, 1>, kBS, L, 1);                          \
  grid_for((const void*)k_pre_s<T>, kBS, L, 1);                          \
  grid_for((const void*)k_upd<T>, 256, L, 1);                            \
  grid_for((const void*)k_matvec_hat<T>, kBS, L, 1);                     \
  grid_for((const void*)k_tinv<T>, kBS, L, 1);                           \
  grid_for((const void*)k_hmv<T>, kBS, L, 1);
  HZ_WARM(float)
  HZ_WARM(double)
#undef HZ_WARM
  warm_launch_kernels(L);
}

}  // namespace hz
