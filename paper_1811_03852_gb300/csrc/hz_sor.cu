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
#include "hz_krylov.cuh"

namespace hz {

namespace {

struct Rb {
  int nx, ny, nz, hx;
  int64_t ncol, H;
};

__device__ __forceinline__ Rb make_rb(const Grid& g) { return Rb{g.nx, g.ny, g.nz, g.nx / 2, g.ncol, g.ncol / 2}; }

// compact neighbours of compact column q: e/w/n/s absolute compact columns
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
  const int64_t o = (int64_t)(c ^ 1) * rb.H;
  RbNbr n;
  n.e = o + (int64_t)j * rb.hx + (iE >> 1);
  n.w = o + (int64_t)j * rb.hx + (iW >> 1);
  n.hn = j + 1 < rb.ny;
  n.hs = j > 0;
  n.n = n.hn ? o + (int64_t)(j + 1) * rb.hx + (i >> 1) : 0;
  n.s = n.hs ? o + (int64_t)(j - 1) * rb.hx + (i >> 1) : 0;
  return n;
}

// (Ahat x)_(k, q) in compact order, all six bands
template <typename T>
__device__ __forceinline__ T ahat_rb(const Rb& rb, const Bands<T>& a, const T* x, int64_t q, int k, const RbNbr& nb) {
  const int64_t kk = (int64_t)k * rb.ncol;
  const int64_t idx = kk + q;
  T y = x[idx];
  y = fma(a.E[idx], x[kk + nb.e], y);
  y = fma(a.W[idx], x[kk + nb.w], y);
  if (nb.hn) y = fma(a.N[idx], x[kk + nb.n], y);
  if (nb.hs) y = fma(a.S[idx], x[kk + nb.s], y);
  if (k + 1 < rb.nz) y = fma(a.U[idx], x[idx + rb.ncol], y);
  if (k > 0) y = fma(a.D[idx], x[idx - rb.ncol], y);
  return y;
}

// Thomas back sweep of one column whose forward values y are parked in z:
// z_k = (1 - omega) zold_k + omega (y_k - c'_k x_(k+1)), x the unrelaxed solution.
template <typename T>
__device__ __forceinline__ void back_relax(const Rb& rb, const T* __restrict__ cp, const T* zold, T* z, int64_t q,
                                           T omega, T keep) {
  T xn = T(0);
#pragma unroll 4
  for (int k = rb.nz - 1; k >= 0; --k) {
    const int64_t idx = (int64_t)k * rb.ncol + q;
    const T x = fma(-cp[idx], xn, z[idx]);
    xn = x;
    z[idx] = zold ? fma(keep, zold[idx], omega * x) : omega * x;
  }
}

// Restart of one compact column (rare, out of line): r = rhs - Ahat x,
// r0 = r, p = r.  Returns <r, r> of the column.
template <typename T>
__device__ __noinline__ double restart_rb(const Rb& rb, const Bands<T>& a, const Vecs<T>& w, int64_t q, bool xzero) {
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
    for (int k = 0; k < g.nz; ++k) {
      const int64_t kk = (int64_t)k * g.ncol;
      if (TO_COMPACT)
        dst[kk + q] = src[kk + col];
      else
        dst[kk + col] = src[kk + q];
    }
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
template <typename T, int MODE>
__global__ void __launch_bounds__(kBS, 4) k_sor_first(Grid g, Bands<T> a, Vecs<T> w, T* z1, double omega_d, Ctl* ctl,
                                                      Red red) {
  const Rb rb = make_rb(g);
  bool restart = false, fresh = false, xzero = true;
  T beta = T(0), om = T(0), alpha = T(0);
  if (MODE == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->bodies += 1;  // read only by k_upd, a later launch
    const int state = ctl->state;
    restart = (state == ST_RESTART);
    if (!restart && state != ST_RUNNING) return;
    fresh = ctl->fresh != 0;
    xzero = ctl->xzero != 0;
    beta = (T)ctl->beta;
    om = (T)ctl->omega;
  } else {
    if (ctl->state != ST_RUNNING) return;
    alpha = (T)ctl->alpha;
  }
  const T* __restrict__ rin = ctl->rsel ? w.r : w.rhs;
  T* out = MODE == 0 ? w.p : w.s;  // may be w.p, read above
  const T omega = (T)omega_d;
  double acc = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * kBS + threadIdx.x; q < rb.ncol; q += (int64_t)gridDim.x * kBS) {
    const bool red_col = q < rb.H;
    if (MODE == 0 && restart) {
      acc += restart_rb<T>(rb, a, w, q, xzero);
      if (red_col) {  // forward sweep on the p just written
        T yp = T(0);
        for (int k = 0; k < rb.nz; ++k) {
          const int64_t idx = (int64_t)k * rb.ncol + q;
          yp = fma(a.m[idx], w.p[idx], -a.l[idx] * yp);
          z1[idx] = yp;
        }
      }
    } else {
      T part = T(0), yp = T(0);
#pragma unroll 4
      for (int k = 0; k < rb.nz; ++k) {
        const int64_t idx = (int64_t)k * rb.ncol + q;
        T v;
        if (MODE == 0)
          v = fresh ? rin[idx] : fma(beta, fma(-om, w.v[idx], w.p[idx]), rin[idx]);
        else
          v = fma(-alpha, w.v[idx], rin[idx]);
        out[idx] = v;
        if (MODE == 1) part = fma(v, v, part);
        if (red_col) {
          yp = fma(a.m[idx], v, -a.l[idx] * yp);
          z1[idx] = yp;
        }
      }
      acc += (double)part;
    }
    if (red_col) back_relax<T>(rb, a.cp, (const T*)nullptr, z1, q, omega, T(0));
  }
  if (MODE == 0 && restart) {
    double vv[1] = {acc}, o[1];
    if (grid_reduce<1>(vv, red, o)) fin_restart(ctl, o[0]);
  } else if (MODE == 1) {
    double vv[1] = {acc}, o[1];
    if (grid_reduce<1>(vv, red, o)) fin_snorm(ctl, o[0]);
  }
}

// One colour pass: for every column of the colour,
//   zout = (1 - omega) zold + omega T^-1 (rc - H znbr),
// H the four horizontal bands (their neighbours all have the other colour).
// zold == nullptr: the first sweep (previous iterate zero).  nbr == 0: the
// other colour is still zero (the red pass of the first sweep).  znbr and zout
// may be the same buffer (different halves).  ctl (may be null): nothing to do
// unless the inner solve is running.
template <typename T>
__global__ void __launch_bounds__(kBS, kMinBlocks) k_sor_pass(Grid g, Bands<T> a, const T* __restrict__ rc,
                                                              const T* znbr, const T* zold, T* zout, int colour,
                                                              int nbr, double omega_d, const Ctl* ctl) {
  if (ctl && ctl->state != ST_RUNNING) return;
  const Rb rb = make_rb(g);
  const T omega = (T)omega_d, keep = (T)(1.0 - omega_d);
  for (int64_t h = (int64_t)blockIdx.x * kBS + threadIdx.x; h < rb.H; h += (int64_t)gridDim.x * kBS) {
    const int64_t q = (int64_t)colour * rb.H + h;
    const RbNbr nb = rb_nbr(rb, q);
    T yp = T(0);
#pragma unroll 4
    for (int k = 0; k < rb.nz; ++k) {
      const int64_t kk = (int64_t)k * rb.ncol;
      const int64_t idx = kk + q;
      T rhs = rc[idx];
      if (nbr) {
        T hsum = a.E[idx] * znbr[kk + nb.e];
        hsum = fma(a.W[idx], znbr[kk + nb.w], hsum);
        if (nb.hn) hsum = fma(a.N[idx], znbr[kk + nb.n], hsum);
        if (nb.hs) hsum = fma(a.S[idx], znbr[kk + nb.s], hsum);
        rhs -= hsum;
      }
      yp = fma(a.m[idx], rhs, -a.l[idx] * yp);
      zout[idx] = yp;
    }
    back_relax<T>(rb, a.cp, zold, zout, q, omega, keep);
  }
}

// y = Ahat x in compact order with the iteration's dots:
// MODE 0 (x = ph, y = v): <r0, v> -> alpha;  MODE 1 (x = sh, y = t): <t, s>, <t, t> -> omega
template <typename T, int MODE>
__global__ void __launch_bounds__(kBS, kMinBlocks) k_mv_rb(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl, Red red) {
  if (ctl->state != ST_RUNNING) return;
  const Rb rb = make_rb(g);
  const T* __restrict__ x = MODE == 0 ? w.ph : w.sh;
  T* __restrict__ y = MODE == 0 ? w.v : w.t;
  const T* __restrict__ c = MODE == 0 ? (ctl->r0sel ? w.r0 : w.rhs) : w.s;
  double acc0 = 0.0, acc1 = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * kBS + threadIdx.x; q < rb.ncol; q += (int64_t)gridDim.x * kBS) {
    const RbNbr nb = rb_nbr(rb, q);
    T a0 = T(0), a1 = T(0);
#pragma unroll 4
    for (int k = 0; k < rb.nz; ++k) {
      const int64_t idx = (int64_t)k * rb.ncol + q;
      const T yy = ahat_rb(rb, a, x, q, k, nb);
      y[idx] = yy;
      a0 = fma(c[idx], yy, a0);
      if (MODE == 1) a1 = fma(yy, yy, a1);
    }
    acc0 += (double)a0;
    acc1 += (double)a1;
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
  if (mode == 0)
    k_sor_first<T, 0><<<grid_for((const void*)k_sor_first<T, 0>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, z1,
                                                                                                        omega, ctl, red);
  else
    k_sor_first<T, 1><<<grid_for((const void*)k_sor_first<T, 1>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, z1,
                                                                                                        omega, ctl, red);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sor_pass(const Grid& g, const Bands<T>& a, const T* rc, const T* znbr, const T* zold, T* zout,
                            int colour, int nbr, double omega, const Ctl* ctl, const Launch& L) {
  const int64_t wb = (g.ncol / 2 + kBS - 1) / kBS;
  k_sor_pass<T><<<grid_for((const void*)k_sor_pass<T>, kBS, L, wb), kBS, 0, L.stream>>>(g, a, rc, znbr, zold, zout,
                                                                                          colour, nbr, omega, ctl);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mv_rb(const Grid& g, const Bands<T>& a, const Vecs<T>& w, int mode, Ctl* ctl, Red red,
                         const Launch& L) {
  if (mode == 0)
    k_mv_rb<T, 0><<<grid_for((const void*)k_mv_rb<T, 0>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, ctl, red);
  else
    k_mv_rb<T, 1><<<grid_for((const void*)k_mv_rb<T, 1>, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, a, w, ctl, red);
  return cudaGetLastError();
}

template <typename T>
void warm_sor(const Launch& L) {
  grid_for((const void*)k_rb_copy<T, true>, kBS, L, 1);
  grid_for((const void*)k_rb_copy<T, false>, kBS, L, 1);
  grid_for((const void*)k_sor_first<T, 0>, kBS, L, 1);
  grid_for((const void*)k_sor_first<T, 1>, kBS, L, 1);
  grid_for((const void*)k_sor_pass<T>, kBS, L, 1);
  grid_for((const void*)k_mv_rb<T, 0>, kBS, L, 1);
  grid_for((const void*)k_mv_rb<T, 1>, kBS, L, 1);
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
