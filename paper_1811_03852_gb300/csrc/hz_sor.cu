// hz_sor.cu -- the paper's tri-SOR preconditioner on sm_103a.
//
// Maynard & Walters Sec. 2: Ahat = L + T + U with T the vertical tridiagonal
// part; the preconditioner is a few (typically three) sweeps of the
// relaxation
//   x_n = (1 - omega) x_(n-1) + omega T^-1 (r - L x_n - U x_(n-1)),  omega = 1.5,
// from x_0 = 0.  Columns are taken in red-black order (colour (i + j) mod 2,
// red = 0 first; nx must be even so that the periodic east-west neighbour has
// the other colour), so in one colour pass every column reads only the other
// colour and the columns are independent.
//
// Layout.  With this preconditioner the whole inner solve runs in
// colour-compact column order, c = colour * (ncol/2) + j * (nx/2) + i/2: the
// six scaled bands and the Thomas factors are permuted once per operator, the
// inner right-hand side is gathered into this order and the inner solution
// scattered back around every refinement step (the FP64 residual stays in
// natural order).  A colour pass then streams one contiguous half of every
// array, and the E/W/N/S neighbours of a compact column are at compact
// columns of the other half that stay contiguous across a warp.  Inner
// products and the elementwise BiCGStab updates are unchanged by the
// relabelling.
//
// Sweeps ping-pong between two buffers: a pass reads the other colour's
// newest values and its own previous values from one buffer and writes its
// colour to the other, so the forward Thomas sweep can park y in the output
// column (as the T^-1 kernels do) and no extra array is needed.
//
// Every column march is software-pipelined like the T^-1 kernels: the loads
// of U levels are issued before any of them is used (U from 1 to 4 by kernel
// and precision, the largest that keeps the kernel within 80 registers
// without spilling).
#include "hz_krylov.cuh"

namespace hz {

namespace {

struct Rb {
  int nx, ny, nz, hx;
  int64_t ncol, H;
};

__device__ __forceinline__ Rb make_rb(const Grid& g) { return Rb{g.nx, g.ny, g.nz, g.nx / 2, g.ncol, g.ncol / 2}; }

// neighbours of compact column q, as offsets from q (the same at every level)
struct RbNbr {
  int64_t e, w, n, s;
  bool hn, hs;
};

__device__ __forceinline__ RbNbr rb_nbr(const Rb& rb, int64_t q) {
  const int c = q >= rb.H ? 1 : 0;
  const int64_t r = q - (int64_t)c * rb.H;
  const int j = (int)(r / rb.hx);
  const int qi = (int)(r - (int64_t)j * rb.hx);
  const int i = 2 * qi + ((j + c) & 1);
  const int iE = (i + 1 == rb.nx) ? 0 : i + 1;
  const int iW = (i == 0) ? rb.nx - 1 : i - 1;
  const int64_t o = (int64_t)(c ^ 1) * rb.H - q;
  RbNbr n;
  n.e = o + (int64_t)j * rb.hx + (iE >> 1);
  n.w = o + (int64_t)j * rb.hx + (iW >> 1);
  n.hn = j + 1 < rb.ny;
  n.hs = j > 0;
  n.n = n.hn ? o + (int64_t)(j + 1) * rb.hx + (i >> 1) : 0;
  n.s = n.hs ? o + (int64_t)(j - 1) * rb.hx + (i >> 1) : 0;
  return n;
}

// Work items of a kernel over both colours: item w maps to blocks of kBS red
// and kBS black columns in turn, so that the blocks resident at one time
// cover the same rows of both halves (a column read as the other colour's
// neighbour is then still in L2 from its own read).  rb_col returns -1 for
// the padding items past the end of a half.
__device__ __forceinline__ int64_t rb_items(const Rb& rb) { return 2 * ((rb.H + kBS - 1) / kBS) * kBS; }
__device__ __forceinline__ int64_t rb_col(const Rb& rb, int64_t w) {
  const int64_t pb = w / (2 * kBS);
  const int within = (int)(w - pb * 2 * kBS);
  const int colour = within >= kBS ? 1 : 0;
  const int64_t off = pb * kBS + (within - colour * kBS);
  return off < rb.H ? (int64_t)colour * rb.H + off : -1;
}

// (Ahat x)_(k, q) in compact order, all six bands (restart path only)
template <typename T>
__device__ __forceinline__ T ahat_rb(const Rb& rb, const Bands<T>& a, const T* x, int64_t q, int k, const RbNbr& nb) {
  const int64_t idx = (int64_t)k * rb.ncol + q;
  T y = x[idx];
  y = fma(a.E[idx], x[idx + nb.e], y);
  y = fma(a.W[idx], x[idx + nb.w], y);
  if (nb.hn) y = fma(a.N[idx], x[idx + nb.n], y);
  if (nb.hs) y = fma(a.S[idx], x[idx + nb.s], y);
  if (k + 1 < rb.nz) y = fma(a.U[idx], x[idx + rb.ncol], y);
  if (k > 0) y = fma(a.D[idx], x[idx - rb.ncol], y);
  return y;
}

// Relaxed Thomas solve of one column with unit diagonal and pre-computed
// factors: forward y_k = m_k q_k - l_k y_(k-1) with q_k = src.make(...), y
// parked in z; back x_k = y_k - c'_k x_(k+1) and
// z_k = (1 - omega) zold_k + omega x_k (zold == nullptr: zero).
template <typename T, int U, typename Src>
__device__ __forceinline__ void sor_column(const Rb& rb, int64_t q, const T* __restrict__ m, const T* __restrict__ l,
                                           const T* __restrict__ cp, const T* __restrict__ zold, T* __restrict__ z,
                                           T omega, T keep, Src& src) {
  constexpr int NIN = Src::NIN;
  const int64_t ncol = rb.ncol;
  const int nz = rb.nz;
  T yprev = T(0);
  for (int k0 = 0; k0 < nz; k0 += U) {
    T v[U][NIN], mm[U], ll[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + q;
        src.load(idx, v[u]);
        mm[u] = __ldg(m + idx);
        ll[u] = __ldg(l + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + q;
        const T qv = src.make(v[u], idx);
        yprev = fma(mm[u], qv, -ll[u] * yprev);
        z[idx] = yprev;
      }
    }
    src.flush();
  }
  T xn = T(0);
  for (int k0 = nz - 1; k0 >= 0; k0 -= 2 * U) {
    T yy[2 * U], cc[2 * U], zo[2 * U];
#pragma unroll
    for (int u = 0; u < 2 * U; ++u) {
      if (k0 - u >= 0) {
        const int64_t idx = (int64_t)(k0 - u) * ncol + q;
        yy[u] = z[idx];  // written by this thread above: coherent load
        cc[u] = __ldg(cp + idx);
        zo[u] = zold ? __ldg(zold + idx) : T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < 2 * U; ++u) {
      if (k0 - u >= 0) {
        const int64_t idx = (int64_t)(k0 - u) * ncol + q;
        xn = fma(-cc[u], xn, yy[u]);
        z[idx] = fma(keep, zo[u], omega * xn);
      }
    }
  }
}

// inputs of the relaxed solves ------------------------------------------------
template <typename T>
struct SrcHz {  // q = rc - (E zE + W zW + N zN + S zS); nbr == false: q = rc
  static constexpr int NIN = 9;
  const T* __restrict__ rc;
  const T* __restrict__ E;
  const T* __restrict__ W;
  const T* __restrict__ N;
  const T* __restrict__ S;
  const T* __restrict__ zn;  // other colour's newest values (read-only in the pass)
  RbNbr nb;
  bool nbr;
  __device__ __forceinline__ void load(int64_t idx, T (&o)[NIN]) {
    o[0] = __ldg(rc + idx);
    if (nbr) {
      o[1] = __ldg(E + idx);
      o[2] = __ldg(zn + idx + nb.e);
      o[3] = __ldg(W + idx);
      o[4] = __ldg(zn + idx + nb.w);
      o[5] = nb.hn ? __ldg(N + idx) : T(0);
      o[6] = nb.hn ? __ldg(zn + idx + nb.n) : T(0);
      o[7] = nb.hs ? __ldg(S + idx) : T(0);
      o[8] = nb.hs ? __ldg(zn + idx + nb.s) : T(0);
    }
  }
  __device__ __forceinline__ T make(const T (&o)[NIN], int64_t) {
    if (!nbr) return o[0];
    T h = o[1] * o[2];
    h = fma(o[3], o[4], h);
    h = fma(o[5], o[6], h);
    h = fma(o[7], o[8], h);
    return o[0] - h;
  }
  __device__ __forceinline__ void flush() {}
};

template <typename T>
struct SrcPu {  // p = r + beta (p - omega v) (fresh: p = r), stored
  static constexpr int NIN = 3;
  const T* __restrict__ r;
  T* __restrict__ p;
  const T* __restrict__ v;
  T beta, omega;
  bool fresh;
  __device__ __forceinline__ void load(int64_t idx, T (&o)[NIN]) {
    o[0] = __ldg(r + idx);
    if (!fresh) {
      o[1] = p[idx];
      o[2] = __ldg(v + idx);
    }
  }
  __device__ __forceinline__ T make(const T (&o)[NIN], int64_t idx) {
    const T q = fresh ? o[0] : fma(beta, fma(-omega, o[2], o[1]), o[0]);
    p[idx] = q;
    return q;
  }
  __device__ __forceinline__ void flush() {}
};

template <typename T>
struct SrcSu {  // s = r - alpha v, stored, with <s, s> (FP32 within a batch, FP64 across)
  static constexpr int NIN = 2;
  const T* __restrict__ r;
  const T* __restrict__ v;
  T* __restrict__ s;
  T alpha;
  T part;
  double acc;
  __device__ __forceinline__ void load(int64_t idx, T (&o)[NIN]) {
    o[0] = __ldg(r + idx);
    o[1] = __ldg(v + idx);
  }
  __device__ __forceinline__ T make(const T (&o)[NIN], int64_t idx) {
    const T q = fma(-alpha, o[1], o[0]);
    s[idx] = q;
    part = fma(q, q, part);
    return q;
  }
  __device__ __forceinline__ void flush() {
    acc += (double)part;
    part = T(0);
  }
};

// the vector update alone on a column (black half of k_sor_first)
template <typename T, int U, typename Src>
__device__ __forceinline__ void update_column(const Rb& rb, int64_t q, Src& src) {
  constexpr int NIN = Src::NIN;
  for (int k0 = 0; k0 < rb.nz; k0 += 2 * U) {
    T v[2 * U][NIN];
#pragma unroll
    for (int u = 0; u < 2 * U; ++u)
      if (k0 + u < rb.nz) src.load((int64_t)(k0 + u) * rb.ncol + q, v[u]);
#pragma unroll
    for (int u = 0; u < 2 * U; ++u)
      if (k0 + u < rb.nz) src.make(v[u], (int64_t)(k0 + u) * rb.ncol + q);
    src.flush();
  }
}

// Restart of one compact column (rare, out of line): r = rhs - Ahat x,
// r0 = r, p = r, and for a red column z1 = omega T^-1 p.  Returns <r, r>.
template <typename T>
__device__ __noinline__ double restart_rb(const Rb& rb, const Bands<T>& a, const Vecs<T>& w, int64_t q, bool xzero,
                                          T* z1, T omega) {
  const RbNbr nb = rb_nbr(rb, q);
  T acc = T(0);
  for (int k = 0; k < rb.nz; ++k) {
    const int64_t idx = (int64_t)k * rb.ncol + q;
    T v = w.rhs[idx];
    if (!xzero) v -= ahat_rb(rb, a, w.x, q, k, nb);
    w.r[idx] = v;
    w.r0[idx] = v;
    w.p[idx] = v;
    acc = fma(v, v, acc);
  }
  if (q < rb.H) {
    T yp = T(0);
    for (int k = 0; k < rb.nz; ++k) {
      const int64_t idx = (int64_t)k * rb.ncol + q;
      yp = fma(a.m[idx], w.p[idx], -a.l[idx] * yp);
      z1[idx] = yp;
    }
    T xn = T(0);
    for (int k = rb.nz - 1; k >= 0; --k) {
      const int64_t idx = (int64_t)k * rb.ncol + q;
      xn = fma(-a.cp[idx], xn, z1[idx]);
      z1[idx] = omega * xn;
    }
  }
  return (double)acc;
}

}  // namespace

// ---------------------------------------------------------------------------
// natural <-> compact copies (one thread per natural column: the natural side
// is read or written contiguously, the compact side in two contiguous halves)
template <typename T, bool TO_COMPACT>
__global__ void __launch_bounds__(kBS) k_rb_copy(Grid g, const T* __restrict__ src, T* __restrict__ dst) {
  const int hx = g.nx / 2;
  const int64_t H = g.ncol / 2;
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    const int i = (int)(col % g.nx), j = (int)(col / g.nx);
    const int64_t q = (int64_t)((i + j) & 1) * H + (int64_t)j * hx + (i >> 1);
    constexpr int B = 8;
    for (int k0 = 0; k0 < g.nz; k0 += B) {
      T v[B];
#pragma unroll
      for (int u = 0; u < B; ++u)
        if (k0 + u < g.nz) v[u] = __ldg(src + (int64_t)(k0 + u) * g.ncol + (TO_COMPACT ? col : q));
#pragma unroll
      for (int u = 0; u < B; ++u)
        if (k0 + u < g.nz) dst[(int64_t)(k0 + u) * g.ncol + (TO_COMPACT ? q : col)] = v[u];
    }
  }
}

// ---------------------------------------------------------------------------
// Variants (the autotuner picks one per kernel, precision and grid): U levels
// per batch and MINB blocks per SM (the register budget).  Each table lists
// only shapes that compile without spills.
template <typename T>
struct SorVar;
template <>
struct SorVar<float> {
  static constexpr int NK[3] = {4, 3, 3};
  static constexpr int u[3][4] = {{2, 4, 1, 3}, {4, 2, 8, 0}, {4, 2, 3, 0}};
  static constexpr int b[3][4] = {{6, 4, 8, 5}, {6, 8, 4, 0}, {6, 8, 5, 0}};
};
template <>
struct SorVar<double> {
  static constexpr int NK[3] = {3, 3, 3};
  static constexpr int u[3][4] = {{1, 2, 2, 0}, {1, 2, 1, 0}, {1, 2, 1, 0}};
  static constexpr int b[3][4] = {{6, 4, 5, 0}, {6, 4, 8, 0}, {6, 4, 8, 0}};
};

template <typename T, int KIND, int I = 0, typename F>
cudaError_t with_sor(int id, F&& f) {
  if constexpr (I < SorVar<T>::NK[KIND]) {
    if (id == I)
      return f(std::integral_constant<int, SorVar<T>::u[KIND][I]>{}, std::integral_constant<int, SorVar<T>::b[KIND][I]>{});
    return with_sor<T, KIND, I + 1>(id, f);
  } else {
    return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// k_sor_first<0>: p = r + beta (p - omega v) (p = r after a start; on a
//   restart, Sec. 4: r = rhs - Ahat x, r0 = r, p = r and ||r||^2), then the red
//   pass of the first sweep on the new p: z1 = omega T^-1 p on red columns.
// k_sor_first<1>: s = r - alpha v, ||s||^2 (half-step exit test), then the
//   same first red pass on s.
// All columns are updated; only the red half (compact columns < ncol/2)
// continues into the tridiagonal solve.
template <typename T, int MODE, int U, int MINB>
__global__ void __launch_bounds__(kBS, MINB) k_sor_first(Grid g, Bands<T> a, Vecs<T> w, T* __restrict__ z1,
                                                         double omega_d, Ctl* ctl, Red red) {
  const Rb rb = make_rb(g);
  bool restart = false;
  if (MODE == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->bodies += 1;  // read only by k_upd, a later launch
    const int state = ctl->state;
    restart = (state == ST_RESTART);
    if (!restart && state != ST_RUNNING) return;
  } else {
    if (ctl->state != ST_RUNNING) return;
  }
  const T* rin = ctl->rsel ? w.r : w.rhs;
  const T omega = (T)omega_d;
  double acc = 0.0;
  if (MODE == 0 && restart) {
    const bool xzero = ctl->xzero != 0;
    for (int64_t q = (int64_t)blockIdx.x * kBS + threadIdx.x; q < rb.ncol; q += (int64_t)gridDim.x * kBS)
      acc += restart_rb<T>(rb, a, w, q, xzero, z1, omega);
    double vv[1] = {acc}, o[1];
    if (grid_reduce<1>(vv, red, o)) fin_restart(ctl, o[0]);
    return;
  }
  const int64_t items = rb_items(rb);
  if (MODE == 0) {
    SrcPu<T> src{rin, w.p, w.v, (T)ctl->beta, (T)ctl->omega, ctl->fresh != 0};
    for (int64_t it = (int64_t)blockIdx.x * kBS + threadIdx.x; it < items; it += (int64_t)gridDim.x * kBS) {
      const int64_t q = rb_col(rb, it);
      if (q < 0) continue;
      if (q < rb.H)
        sor_column<T, U>(rb, q, a.m, a.l, a.cp, nullptr, z1, omega, T(0), src);
      else
        update_column<T, U>(rb, q, src);
    }
  } else {
    SrcSu<T> src{rin, w.v, w.s, (T)ctl->alpha, T(0), 0.0};
    for (int64_t it = (int64_t)blockIdx.x * kBS + threadIdx.x; it < items; it += (int64_t)gridDim.x * kBS) {
      const int64_t q = rb_col(rb, it);
      if (q < 0) continue;
      if (q < rb.H)
        sor_column<T, U>(rb, q, a.m, a.l, a.cp, nullptr, z1, omega, T(0), src);
      else
        update_column<T, U>(rb, q, src);
    }
    double vv[1] = {src.acc}, o[1];
    if (grid_reduce<1>(vv, red, o)) fin_snorm(ctl, o[0]);
  }
}

// One colour pass: for every column of the colour,
//   zout = (1 - omega) zold + omega T^-1 (rc - H znbr),
// H the four horizontal bands (their neighbours all have the other colour).
// zold == nullptr: the first sweep (previous iterate zero).  nbr == 0: the
// other colour is still zero (the red pass of the first sweep).  znbr and zout
// may be the same buffer: the pass reads only the other colour's half of it
// and writes only its own.  ctl (may be null): nothing to do unless the inner
// solve is running.
template <typename T, int U, int MINB>
__global__ void __launch_bounds__(kBS, MINB) k_sor_pass(Grid g, Bands<T> a, const T* __restrict__ rc,
                                                        const T* __restrict__ znbr, const T* __restrict__ zold,
                                                        T* __restrict__ zout, int colour, int nbr, double omega_d,
                                                        const Ctl* ctl) {
  if (ctl && ctl->state != ST_RUNNING) return;
  const Rb rb = make_rb(g);
  const T omega = (T)omega_d, keep = (T)(1.0 - omega_d);
  for (int64_t h = (int64_t)blockIdx.x * kBS + threadIdx.x; h < rb.H; h += (int64_t)gridDim.x * kBS) {
    const int64_t q = (int64_t)colour * rb.H + h;
    SrcHz<T> src{rc, a.E, a.W, a.N, a.S, znbr, rb_nbr(rb, q), nbr != 0};
    sor_column<T, U>(rb, q, a.m, a.l, a.cp, zold, zout, omega, keep, src);
  }
}

// y = Ahat x in compact order with the iteration's dots:
// MODE 0 (x = ph, y = v): <r0, v> -> alpha;  MODE 1 (x = sh, y = t): <t, s>, <t, t> -> omega.
// The column's own values ride down in registers (x_(k-1), x_k); each level
// loads x_(k+1), the four horizontal neighbours, six bands and the dot partner.
template <typename T, int MODE, int U, int MINB>
__global__ void __launch_bounds__(kBS, MINB) k_mv_rb(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl, Red red) {
  if (ctl->state != ST_RUNNING) return;
  const Rb rb = make_rb(g);
  const T* __restrict__ x = MODE == 0 ? w.ph : w.sh;
  T* __restrict__ y = MODE == 0 ? w.v : w.t;
  const T* __restrict__ c = MODE == 0 ? (ctl->r0sel ? w.r0 : w.rhs) : w.s;
  const T* __restrict__ E = a.E;
  const T* __restrict__ W = a.W;
  const T* __restrict__ N = a.N;
  const T* __restrict__ S = a.S;
  const T* __restrict__ Up = a.U;
  const T* __restrict__ Dn = a.D;
  const int64_t ncol = rb.ncol;
  const int nz = rb.nz;
  double acc0 = 0.0, acc1 = 0.0;
  const int64_t items = rb_items(rb);
  for (int64_t it = (int64_t)blockIdx.x * kBS + threadIdx.x; it < items; it += (int64_t)gridDim.x * kBS) {
    const int64_t q = rb_col(rb, it);
    if (q < 0) continue;
    const RbNbr nb = rb_nbr(rb, q);
    T xm = T(0), x0 = __ldg(x + q);
    for (int k0 = 0; k0 < nz; k0 += U) {
      T xp[U], he[U], hw[U], hn[U], hs[U], be[U], bw[U], bn[U], bs[U], bu[U], bd[U], cc[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + u;
        if (k < nz) {
          const int64_t idx = (int64_t)k * ncol + q;
          xp[u] = k + 1 < nz ? __ldg(x + idx + ncol) : T(0);
          he[u] = __ldg(x + idx + nb.e);
          hw[u] = __ldg(x + idx + nb.w);
          hn[u] = nb.hn ? __ldg(x + idx + nb.n) : T(0);
          hs[u] = nb.hs ? __ldg(x + idx + nb.s) : T(0);
          be[u] = __ldg(E + idx);
          bw[u] = __ldg(W + idx);
          bn[u] = nb.hn ? __ldg(N + idx) : T(0);
          bs[u] = nb.hs ? __ldg(S + idx) : T(0);
          bu[u] = __ldg(Up + idx);
          bd[u] = __ldg(Dn + idx);
          cc[u] = __ldg(c + idx);
        }
      }
      T a0 = T(0), a1 = T(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + u;
        if (k < nz) {
          T yy = x0;
          yy = fma(be[u], he[u], yy);
          yy = fma(bw[u], hw[u], yy);
          yy = fma(bn[u], hn[u], yy);
          yy = fma(bs[u], hs[u], yy);
          yy = fma(bu[u], xp[u], yy);
          yy = fma(bd[u], xm, yy);
          y[(int64_t)k * ncol + q] = yy;
          a0 = fma(cc[u], yy, a0);
          if (MODE == 1) a1 = fma(yy, yy, a1);
          xm = x0;
          x0 = xp[u];
        }
      }
      acc0 += (double)a0;
      acc1 += (double)a1;
    }
  }
  if (MODE == 0) {
    double vv[1] = {acc0}, o[1];
    if (grid_reduce<1>(vv, red, o)) fin_alpha(ctl, o[0]);
  } else {
    double vv[2] = {acc0, acc1}, o[2];
    if (grid_reduce<2>(vv, red, o)) fin_omega(ctl, o[0], o[1]);
  }
}

// ---------------------------------------------------------------------------
template <typename T>
constexpr int sor_prec() {
  return sizeof(T) == 8 ? 1 : 0;
}

template <typename T>
cudaError_t launch_rb_copy(const Grid& g, const T* src, T* dst, int to_compact, const Launch& L) {
  if (to_compact)
    k_rb_copy<T, true><<<grid_for((const void*)k_rb_copy<T, true>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, src, dst);
  else
    k_rb_copy<T, false><<<grid_for((const void*)k_rb_copy<T, false>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, src, dst);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sor_first(const Grid& g, const Bands<T>& a, const Vecs<T>& w, T* z1, double omega, int mode,
                             Ctl* ctl, Red red, const Launch& L) {
  return with_sor<T, 2>(L.vsor[sor_prec<T>()][2], [&](auto uc, auto bc) {
    constexpr int U = decltype(uc)::value, B = decltype(bc)::value;
    if (mode == 0)
      k_sor_first<T, 0, U, B><<<grid_for((const void*)k_sor_first<T, 0, U, B>, kBS, L, L.wcol), kBS, 0, L.stream>>>(
          g, a, w, z1, omega, ctl, red);
    else
      k_sor_first<T, 1, U, B><<<grid_for((const void*)k_sor_first<T, 1, U, B>, kBS, L, L.wcol), kBS, 0, L.stream>>>(
          g, a, w, z1, omega, ctl, red);
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_sor_pass(const Grid& g, const Bands<T>& a, const T* rc, const T* znbr, const T* zold, T* zout,
                            int colour, int nbr, double omega, const Ctl* ctl, const Launch& L) {
  const int64_t wb = (g.ncol / 2 + kBS - 1) / kBS;
  return with_sor<T, 0>(L.vsor[sor_prec<T>()][0], [&](auto uc, auto bc) {
    constexpr int U = decltype(uc)::value, B = decltype(bc)::value;
    k_sor_pass<T, U, B><<<grid_for((const void*)k_sor_pass<T, U, B>, kBS, L, wb), kBS, 0, L.stream>>>(
        g, a, rc, znbr, zold, zout, colour, nbr, omega, ctl);
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_mv_rb(const Grid& g, const Bands<T>& a, const Vecs<T>& w, int mode, Ctl* ctl, Red red,
                         const Launch& L) {
  return with_sor<T, 1>(L.vsor[sor_prec<T>()][1], [&](auto uc, auto bc) {
    constexpr int U = decltype(uc)::value, B = decltype(bc)::value;
    if (mode == 0)
      k_mv_rb<T, 0, U, B><<<grid_for((const void*)k_mv_rb<T, 0, U, B>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w,
                                                                                                            ctl, red);
    else
      k_mv_rb<T, 1, U, B><<<grid_for((const void*)k_mv_rb<T, 1, U, B>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w,
                                                                                                            ctl, red);
    return cudaGetLastError();
  });
}

template <typename T>
void warm_sor(const Launch& L) {
  grid_for((const void*)k_rb_copy<T, true>, kBS, L, 1);
  grid_for((const void*)k_rb_copy<T, false>, kBS, L, 1);
  for (int id = 0; id < SorVar<T>::NK[0]; ++id)
    with_sor<T, 0>(id, [&](auto uc, auto bc) {
      grid_for((const void*)k_sor_pass<T, decltype(uc)::value, decltype(bc)::value>, kBS, L, 1);
      return cudaSuccess;
    });
  for (int id = 0; id < SorVar<T>::NK[1]; ++id)
    with_sor<T, 1>(id, [&](auto uc, auto bc) {
      grid_for((const void*)k_mv_rb<T, 0, decltype(uc)::value, decltype(bc)::value>, kBS, L, 1);
      grid_for((const void*)k_mv_rb<T, 1, decltype(uc)::value, decltype(bc)::value>, kBS, L, 1);
      return cudaSuccess;
    });
  for (int id = 0; id < SorVar<T>::NK[2]; ++id)
    with_sor<T, 2>(id, [&](auto uc, auto bc) {
      grid_for((const void*)k_sor_first<T, 0, decltype(uc)::value, decltype(bc)::value>, kBS, L, 1);
      grid_for((const void*)k_sor_first<T, 1, decltype(uc)::value, decltype(bc)::value>, kBS, L, 1);
      return cudaSuccess;
    });
}

int sor_num_variants(int prec, int kind) {
  if (kind < 0 || kind > 2) return 0;
  return prec == 0 ? SorVar<float>::NK[kind] : SorVar<double>::NK[kind];
}

void sor_variant_shape(int prec, int kind, int id, int* depth, int* minb) {
  *depth = prec == 0 ? SorVar<float>::u[kind][id] : SorVar<double>::u[kind][id];
  *minb = prec == 0 ? SorVar<float>::b[kind][id] : SorVar<double>::b[kind][id];
}

#define HZ_SOR_INST(T)                                                                                               \
  template cudaError_t launch_rb_copy<T>(const Grid&, const T*, T*, int, const Launch&);                           \
  template cudaError_t launch_sor_first<T>(const Grid&, const Bands<T>&, const Vecs<T>&, T*, double, int, Ctl*, Red, \
                                           const Launch&);                                                           \
  template cudaError_t launch_sor_pass<T>(const Grid&, const Bands<T>&, const T*, const T*, const T*, T*, int, int,   \
                                          double, const Ctl*, const Launch&);                                        \
  template cudaError_t launch_mv_rb<T>(const Grid&, const Bands<T>&, const Vecs<T>&, int, Ctl*, Red, const Launch&); \
  template void warm_sor<T>(const Launch&);

HZ_SOR_INST(float)
HZ_SOR_INST(double)

}  // namespace hz
