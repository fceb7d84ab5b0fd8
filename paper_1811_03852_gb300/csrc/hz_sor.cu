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
// colour-compact column order, c = colour * H + j * (nx/2) + i/2 with
// H = ncol/2: the six scaled bands and the Thomas factors are permuted once
// per operator, the inner right-hand side is gathered into this order and the
// inner solution scattered back around every refinement step (the FP64
// residual stays in natural order).  A colour pass then streams one
// contiguous half of every array.  Inner products and the elementwise
// BiCGStab updates are unchanged by the relabelling.
//
// Groups.  A thread owns V consecutive compact columns of one row (V divides
// nx/2) and marches k with V-wide vector loads, U levels per software-
// pipelined batch.  The other colour's values at the same (j, i/2) sit at
// compact offset +-H (the "mirror" group): with p the parity of the first
// column's i, its east neighbours are mirror[c + p] and its west neighbours
// mirror[c + p - 1], so one aligned vector load of the mirror group plus one
// scalar (the west neighbour of column 0 when p = 0, the east neighbour of
// column V-1 when p = 1, wrapping around the periodic row) give all of them;
// north and south are the mirror groups of rows j +- 1 (offset +-nx/2).
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

// other-colour neighbours of the group starting at compact column q0, as
// offsets from the group's own index (the same at every level)
struct RbGrp {
  int64_t mir;  // mirror group: +H (red group) or -H (black group)
  int64_t xo;   // the extra scalar (see above)
  int64_t hx;   // row length of a half (north = mir + hx, south = mir - hx)
  bool p;       // parity of i of the group's first column
  bool hn, hs;  // north / south row exists
};

template <int V>
__device__ __forceinline__ RbGrp rb_grp(const Rb& rb, int64_t q0) {
  const int c = q0 >= rb.H ? 1 : 0;
  const int64_t r = q0 - (int64_t)c * rb.H;
  const int j = (int)(r / rb.hx);
  const int qi = (int)(r - (int64_t)j * rb.hx);
  RbGrp gr;
  gr.mir = c ? -rb.H : rb.H;
  gr.p = ((j + c) & 1) != 0;
  if (!gr.p)
    gr.xo = gr.mir + (qi == 0 ? (int64_t)(rb.hx - 1) : (int64_t)-1);
  else
    gr.xo = gr.mir + (qi + V == rb.hx ? (int64_t)-qi : (int64_t)V);
  gr.hx = rb.hx;
  gr.hn = j + 1 < rb.ny;
  gr.hs = j > 0;
  return gr;
}

// east / west neighbour of column c of the group from the mirror vector m and the extra scalar x
template <typename T, int V>
__device__ __forceinline__ T nbr_e(const RbGrp& gr, const Pack<T, V>& m, T x, int c) {
  if (!gr.p) return m.a[c];
  return c + 1 < V ? m.a[(c + 1) % V] : x;
}
template <typename T, int V>
__device__ __forceinline__ T nbr_w(const RbGrp& gr, const Pack<T, V>& m, T x, int c) {
  if (gr.p) return m.a[c];
  return c > 0 ? m.a[(c + V - 1) % V] : x;
}

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> zero_pack() {
  Pack<T, V> z;
#pragma unroll
  for (int c = 0; c < V; ++c) z.a[c] = T(0);
  return z;
}

// Relaxed Thomas solve of V columns with unit diagonal and pre-computed
// factors: forward y_k = m_k q_k - l_k y_(k-1) with q_k = src.make(...), y
// parked in z; back x_k = y_k - c'_k x_(k+1) and
// z_k = (1 - omega) zold_k + omega x_k (zold == nullptr: zero).
// H: L2 priorities (the arrays read once evict-first, the parked forward
// sweep evict-last so that it is still in L2 for the back sweep).
template <typename T, int V, int U, typename Src, bool H = false>
__device__ __forceinline__ void sor_group(const Rb& rb, int64_t q0, const T* __restrict__ m, const T* __restrict__ l,
                                          const T* __restrict__ cp, const T* __restrict__ zold, T* __restrict__ z,
                                          T omega, T keep, Src& src) {
  constexpr int LF = H ? LD_NC_EF : LD_NC;
  constexpr int SY = H ? ST_EL : ST_PLAIN;
  constexpr int SZ = H ? ST_EF : ST_PLAIN;
  const int64_t ncol = rb.ncol;
  const int nz = rb.nz;
  T yprev[V];
#pragma unroll
  for (int c = 0; c < V; ++c) yprev[c] = T(0);
  for (int k0 = 0; k0 < nz; k0 += U) {
    typename Src::In v[U];
    Pack<T, V> mm[U], ll[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + q0;
        src.load(idx, v[u]);
        mm[u] = ldp<T, V, LF>(m + idx);
        ll[u] = ldp<T, V, LF>(l + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + q0;
        const Pack<T, V> q = src.make(v[u], idx);
        Pack<T, V> y;
#pragma unroll
        for (int c = 0; c < V; ++c) {
          y.a[c] = fma(mm[u].a[c], q.a[c], -ll[u].a[c] * yprev[c]);
          yprev[c] = y.a[c];
        }
        stp<T, V, SY>(z + idx, y);
      }
    }
    src.flush();
  }
  T xn[V];
#pragma unroll
  for (int c = 0; c < V; ++c) xn[c] = T(0);
  constexpr int UB = 2 * U;
  for (int k0 = nz - 1; k0 >= 0; k0 -= UB) {
    Pack<T, V> yy[UB], cc[UB], zo[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      if (k0 - u >= 0) {
        const int64_t idx = (int64_t)(k0 - u) * ncol + q0;
        yy[u] = ldp<T, V, LD_PLAIN>(z + idx);  // written by this thread above: coherent load
        cc[u] = ldp<T, V, LF>(cp + idx);
        zo[u] = zold ? ldp<T, V, LF>(zold + idx) : zero_pack<T, V>();
      }
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
      if (k0 - u >= 0) {
        const int64_t idx = (int64_t)(k0 - u) * ncol + q0;
        Pack<T, V> o;
#pragma unroll
        for (int c = 0; c < V; ++c) {
          xn[c] = fma(-cc[u].a[c], xn[c], yy[u].a[c]);
          o.a[c] = fma(keep, zo[u].a[c], omega * xn[c]);
        }
        stp<T, V, SZ>(z + idx, o);
      }
    }
  }
}

// inputs of the relaxed solves ------------------------------------------------
// EF: the sources' once-read arrays carry the L2 evict-first priority (the
// other colour's z, read again by the neighbouring rows, does not)
template <typename T, int V, bool EF = false>
struct SrcHz {  // q = rc - (E zE + W zW + N zN + S zS); nbr == false: q = rc
  static constexpr int MI = EF ? LD_NC_EF : LD_NC;
  struct In {
    Pack<T, V> rc, e, w, n, s, zm, zn, zs;
    T zx;
  };
  const T* __restrict__ rc;
  const T* __restrict__ E;
  const T* __restrict__ W;
  const T* __restrict__ N;
  const T* __restrict__ S;
  const T* __restrict__ z;  // other colour's newest values (read-only in the pass)
  RbGrp gr;
  bool nbr;
  __device__ __forceinline__ void load(int64_t idx, In& o) {
    o.rc = ldp<T, V, MI>(rc + idx);
    if (nbr) {
      o.e = ldp<T, V, MI>(E + idx);
      o.w = ldp<T, V, MI>(W + idx);
      o.zm = ldp<T, V, LD_NC>(z + idx + gr.mir);
      o.zx = ldw<T, LD_NC>(z + idx + gr.xo);
      if (gr.hn) {
        o.n = ldp<T, V, MI>(N + idx);
        o.zn = ldp<T, V, LD_NC>(z + idx + gr.mir + gr.hx);
      } else {
        o.n = o.zn = zero_pack<T, V>();
      }
      if (gr.hs) {
        o.s = ldp<T, V, MI>(S + idx);
        o.zs = ldp<T, V, LD_NC>(z + idx + gr.mir - gr.hx);
      } else {
        o.s = o.zs = zero_pack<T, V>();
      }
    }
  }
  __device__ __forceinline__ Pack<T, V> make(const In& o, int64_t) {
    if (!nbr) return o.rc;
    Pack<T, V> q;
#pragma unroll
    for (int c = 0; c < V; ++c) {
      T h = o.e.a[c] * nbr_e<T, V>(gr, o.zm, o.zx, c);
      h = fma(o.w.a[c], nbr_w<T, V>(gr, o.zm, o.zx, c), h);
      h = fma(o.n.a[c], o.zn.a[c], h);
      h = fma(o.s.a[c], o.zs.a[c], h);
      q.a[c] = o.rc.a[c] - h;
    }
    return q;
  }
  __device__ __forceinline__ void flush() {}
};

template <typename T, int V, bool EF = false>
struct SrcPu {  // p = r + beta (p - omega v) (fresh: p = r), stored
  static constexpr int MI = EF ? LD_NC_EF : LD_NC, MP = EF ? LD_PLAIN_EF : LD_PLAIN, SO = EF ? ST_EF : ST_PLAIN;
  struct In {
    Pack<T, V> r, p, v;
  };
  const T* __restrict__ r;
  T* __restrict__ p;
  const T* __restrict__ v;
  T beta, omega;
  bool fresh;
  __device__ __forceinline__ void load(int64_t idx, In& o) {
    o.r = ldp<T, V, MI>(r + idx);
    if (!fresh) {
      o.p = ldp<T, V, MP>(p + idx);
      o.v = ldp<T, V, MI>(v + idx);
    }
  }
  __device__ __forceinline__ Pack<T, V> make(const In& o, int64_t idx) {
    Pack<T, V> q;
#pragma unroll
    for (int c = 0; c < V; ++c) q.a[c] = fresh ? o.r.a[c] : fma(beta, fma(-omega, o.v.a[c], o.p.a[c]), o.r.a[c]);
    stp<T, V, SO>(p + idx, q);
    return q;
  }
  __device__ __forceinline__ void flush() {}
};

// DOT: also accumulate <s, s>; the solver's half-step test takes it from
// k_mv_rb<1> instead, which reads s anyway
template <typename T, int V, bool EF = false, bool DOT = true>
struct SrcSu {  // s = r - alpha v, stored, optionally with <s, s> (FP32 within a batch, DotAcc across)
  static constexpr int MI = EF ? LD_NC_EF : LD_NC, SO = EF ? ST_EF : ST_PLAIN;
  struct In {
    Pack<T, V> r, v;
  };
  const T* __restrict__ r;
  const T* __restrict__ v;
  T* __restrict__ s;
  T alpha;
  T part;
  DotAcc<T> acc;
  __device__ __forceinline__ void load(int64_t idx, In& o) {
    o.r = ldp<T, V, MI>(r + idx);
    o.v = ldp<T, V, MI>(v + idx);
  }
  __device__ __forceinline__ Pack<T, V> make(const In& o, int64_t idx) {
    Pack<T, V> q;
#pragma unroll
    for (int c = 0; c < V; ++c) {
      q.a[c] = fma(-alpha, o.v.a[c], o.r.a[c]);
      if constexpr (DOT) part = fma(q.a[c], q.a[c], part);
    }
    stp<T, V, SO>(s + idx, q);
    return q;
  }
  __device__ __forceinline__ void flush() {
    if constexpr (DOT) {
      acc.add(part);
      part = T(0);
    }
  }
};

// the vector update alone on a group (black half of k_sor_first)
template <typename T, int V, int U, typename Src>
__device__ __forceinline__ void update_group(const Rb& rb, int64_t q0, Src& src) {
  constexpr int UB = 2 * U;
  for (int k0 = 0; k0 < rb.nz; k0 += UB) {
    typename Src::In v[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u)
      if (k0 + u < rb.nz) src.load((int64_t)(k0 + u) * rb.ncol + q0, v[u]);
#pragma unroll
    for (int u = 0; u < UB; ++u)
      if (k0 + u < rb.nz) src.make(v[u], (int64_t)(k0 + u) * rb.ncol + q0);
    src.flush();
  }
}

// Work items over both colours, in groups: item w maps to blocks of kBS red
// and kBS black groups in turn, so that the blocks resident at one time cover
// the same rows of both halves (a column read as the other colour's
// neighbour is then still in L2 from its own read).  rb_group returns -1 for
// the padding items past the end of a half.
__device__ __forceinline__ int64_t rb_items(int64_t hg) { return 2 * ((hg + kBS - 1) / kBS) * kBS; }
template <int V>
__device__ __forceinline__ int64_t rb_group(const Rb& rb, int64_t hg, int64_t w) {
  const int64_t pb = w / (2 * kBS);
  const int within = (int)(w - pb * 2 * kBS);
  const int colour = within >= kBS ? 1 : 0;
  const int64_t off = pb * kBS + (within - colour * kBS);
  return off < hg ? (int64_t)colour * rb.H + off * V : -1;
}

// Restart of one compact column (rare, out of line): r = rhs - Ahat x,
// r0 = r, p = r, and for a red column z1 = omega T^-1 p.  Returns <r, r>.
template <typename T>
__device__ __noinline__ double restart_rb(const Rb& rb, const Bands<T>& a, const Vecs<T>& w, int64_t q, bool xzero,
                                          T* z1, T omega, const double* x64) {
  const RbGrp gr = rb_grp<1>(rb, q);
  // x in T, or held in FP64 by the paper's mixed-precision solver (arithmetic in T)
  auto X = [&](int64_t i) -> T { return x64 ? (T)x64[i] : w.x[i]; };
  T acc = T(0);
  for (int k = 0; k < rb.nz; ++k) {
    const int64_t idx = (int64_t)k * rb.ncol + q;
    T v = w.rhs[idx];
    if (!xzero) {
      const T xm = X(idx + gr.mir), xx = X(idx + gr.xo);
      T y = X(idx);
      y = fma(a.E[idx], gr.p ? xx : xm, y);
      y = fma(a.W[idx], gr.p ? xm : xx, y);
      if (gr.hn) y = fma(a.N[idx], X(idx + gr.mir + gr.hx), y);
      if (gr.hs) y = fma(a.S[idx], X(idx + gr.mir - gr.hx), y);
      if (k + 1 < rb.nz) y = fma(a.U[idx], X(idx + rb.ncol), y);
      if (k > 0) y = fma(a.D[idx], X(idx - rb.ncol), y);
      v -= y;
    }
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
// Variants (the autotuner picks one per kernel, precision and grid): V columns
// per thread (V divides nx/2), U levels per batch, MINB blocks per SM (the
// register budget) and h: L2 priorities (once-read arrays evict-first, the
// parked forward sweep evict-last).  Variant 0 of every table has V = 1 (any
// even nx).  The tables list only shapes that compile without spills.
template <typename T>
struct SorVar;
template <>
struct SorVar<float> {
  static constexpr int NK[3] = {9, 8, 6};
  static constexpr int v[3][9] = {{1, 1, 2, 4, 4, 2, 4, 2, 4}, {1, 1, 2, 4, 4, 2, 4, 2}, {1, 2, 4, 2, 4, 2}};
  static constexpr int u[3][9] = {{2, 3, 1, 1, 1, 2, 1, 2, 1}, {4, 2, 2, 1, 2, 2, 1, 1}, {4, 2, 1, 2, 1, 2}};
  static constexpr int b[3][9] = {{6, 5, 6, 6, 5, 4, 5, 4, 6}, {6, 8, 6, 6, 4, 6, 6, 6}, {6, 6, 4, 4, 4, 4}};
  static constexpr int h[3][9] = {{0, 0, 0, 0, 0, 0, 1, 1, 1}, {0, 0, 0, 0, 0, 1, 1, 1}, {0, 0, 0, 0, 1, 1}};
};
template <>
struct SorVar<double> {
  static constexpr int NK[3] = {6, 5, 4};
  static constexpr int v[3][9] = {{1, 1, 2, 2, 2, 2}, {1, 1, 2, 2, 2}, {1, 2, 2, 2}};
  static constexpr int u[3][9] = {{1, 2, 1, 1, 1, 1}, {1, 2, 1, 1, 1}, {1, 1, 1, 1}};
  static constexpr int b[3][9] = {{6, 4, 4, 5, 4, 5}, {6, 4, 6, 4, 6}, {6, 4, 5, 4}};
  static constexpr int h[3][9] = {{0, 0, 0, 0, 1, 1}, {0, 0, 0, 0, 1}, {0, 0, 0, 1}};
};

template <typename T, int KIND, int I = 0, typename F>
cudaError_t with_sor(int id, F&& f) {
  if constexpr (I < SorVar<T>::NK[KIND]) {
    if (id == I)
      return f(std::integral_constant<int, SorVar<T>::v[KIND][I]>{}, std::integral_constant<int, SorVar<T>::u[KIND][I]>{},
               std::integral_constant<int, SorVar<T>::b[KIND][I]>{},
               std::integral_constant<bool, SorVar<T>::h[KIND][I] != 0>{});
    return with_sor<T, KIND, I + 1>(id, f);
  } else {
    return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// k_sor_first<0>: p = r + beta (p - omega v) (p = r after a start; on a
//   restart, Sec. 4: r = rhs - Ahat x, r0 = r, p = r and ||r||^2), then the red
//   pass of the first sweep on the new p: z1 = omega T^-1 p on red columns.
// k_sor_first<1>: s = r - alpha v, then the same first red pass on s (the
//   half-step test on ||s|| follows in k_mv_rb<1>).
// All columns are updated; only the red half (compact columns < H) continues
// into the tridiagonal solve.
template <typename T, int MODE, int V, int U, int MINB, bool H>
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
    const bool f32 = sizeof(T) == 4 && ctl->dot32;
    const double* x64 = sizeof(T) == 4 ? ctl->x64 : nullptr;
    for (int64_t q = (int64_t)blockIdx.x * kBS + threadIdx.x; q < rb.ncol; q += (int64_t)gridDim.x * kBS)
      acc = acc_add(acc, restart_rb<T>(rb, a, w, q, xzero, z1, omega, x64), f32);
    double vv[1] = {acc}, o[1];
    if (grid_reduce<1>(vv, red, o, f32)) fin_restart(ctl, o[0]);
    return;
  }
  const int64_t hg = rb.H / V;
  const int64_t items = rb_items(hg);
  if (MODE == 0) {
    using S = SrcPu<T, V, H>;
    S src{rin, w.p, w.v, (T)ctl->beta, (T)ctl->omega, ctl->fresh != 0};
    for (int64_t it = (int64_t)blockIdx.x * kBS + threadIdx.x; it < items; it += (int64_t)gridDim.x * kBS) {
      const int64_t q0 = rb_group<V>(rb, hg, it);
      if (q0 < 0) continue;
      if (q0 < rb.H)
        sor_group<T, V, U, S, H>(rb, q0, a.m, a.l, a.cp, nullptr, z1, omega, T(0), src);
      else
        update_group<T, V, U>(rb, q0, src);
    }
  } else {
    using S = SrcSu<T, V, H, false>;
    S src{rin, w.v, w.s, (T)ctl->alpha, T(0), {}};
    for (int64_t it = (int64_t)blockIdx.x * kBS + threadIdx.x; it < items; it += (int64_t)gridDim.x * kBS) {
      const int64_t q0 = rb_group<V>(rb, hg, it);
      if (q0 < 0) continue;
      if (q0 < rb.H)
        sor_group<T, V, U, S, H>(rb, q0, a.m, a.l, a.cp, nullptr, z1, omega, T(0), src);
      else
        update_group<T, V, U>(rb, q0, src);
    }
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
template <typename T, int V, int U, int MINB, bool H>
__global__ void __launch_bounds__(kBS, MINB) k_sor_pass(Grid g, Bands<T> a, const T* __restrict__ rc,
                                                        const T* __restrict__ znbr, const T* __restrict__ zold,
                                                        T* __restrict__ zout, int colour, int nbr, double omega_d,
                                                        const Ctl* ctl) {
  if (ctl && ctl->state != ST_RUNNING) return;
  const Rb rb = make_rb(g);
  const T omega = (T)omega_d, keep = (T)(1.0 - omega_d);
  const int64_t hg = rb.H / V;
  for (int64_t h = (int64_t)blockIdx.x * kBS + threadIdx.x; h < hg; h += (int64_t)gridDim.x * kBS) {
    const int64_t q0 = (int64_t)colour * rb.H + h * V;
    using S = SrcHz<T, V, H>;
    S src{rc, a.E, a.W, a.N, a.S, znbr, rb_grp<V>(rb, q0), nbr != 0};
    sor_group<T, V, U, S, H>(rb, q0, a.m, a.l, a.cp, zold, zout, omega, keep, src);
  }
}

// y = Ahat x in compact order with the iteration's dots:
// MODE 0 (x = ph, y = v): <r0, v> -> alpha;  MODE 1 (x = sh, y = t): <t, s>,
// <t, t> and <s, s> -> the half-step exit test on ||s||, then omega.  H: the
// bands and the dot partner (read once) evict-first in L2; x, whose mirror
// groups are read again by the neighbouring rows, keeps the normal priority.
// The group's own values ride down in registers (x_(k-1), x_k); each level
// loads x_(k+1), the mirror groups of rows j-1, j, j+1 and one scalar, six
// bands and the dot partner.
template <typename T, int MODE, int V, int U, int MINB, bool H>
__global__ void __launch_bounds__(kBS, MINB) k_mv_rb(Grid g, Bands<T> a, Vecs<T> w, Ctl* ctl, Red red) {
  if (ctl->state != ST_RUNNING) return;
  constexpr int MB = H ? LD_NC_EF : LD_NC;
  constexpr int SY = H ? ST_EF : ST_PLAIN;
  const Rb rb = make_rb(g);
  const T* __restrict__ x = MODE == 0 ? w.ph : w.sh;
  T* __restrict__ y = MODE == 0 ? w.v : w.t;
  const T* __restrict__ c = MODE == 0 ? (ctl->r0sel ? w.r0 : w.rhs) : w.s;
  const int64_t ncol = rb.ncol;
  const int nz = rb.nz;
  const int64_t hg = rb.H / V;
  DotAcc<T> acc0{}, acc1{}, acc2{};
  const int64_t items = rb_items(hg);
  for (int64_t it = (int64_t)blockIdx.x * kBS + threadIdx.x; it < items; it += (int64_t)gridDim.x * kBS) {
    const int64_t q0 = rb_group<V>(rb, hg, it);
    if (q0 < 0) continue;
    const RbGrp gr = rb_grp<V>(rb, q0);
    Pack<T, V> xm = zero_pack<T, V>(), x0 = ldp<T, V, LD_NC>(x + q0);
    for (int k0 = 0; k0 < nz; k0 += U) {
      Pack<T, V> xp[U], hm[U], hn[U], hs[U], be[U], bw[U], bn[U], bs[U], bu[U], bd[U], cc[U];
      T hx1[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + u;
        if (k < nz) {
          const int64_t idx = (int64_t)k * ncol + q0;
          xp[u] = k + 1 < nz ? ldp<T, V, LD_NC>(x + idx + ncol) : zero_pack<T, V>();
          hm[u] = ldp<T, V, LD_NC>(x + idx + gr.mir);
          hx1[u] = ldw<T, LD_NC>(x + idx + gr.xo);
          be[u] = ldp<T, V, MB>(a.E + idx);
          bw[u] = ldp<T, V, MB>(a.W + idx);
          if (gr.hn) {
            hn[u] = ldp<T, V, LD_NC>(x + idx + gr.mir + gr.hx);
            bn[u] = ldp<T, V, MB>(a.N + idx);
          } else {
            hn[u] = bn[u] = zero_pack<T, V>();
          }
          if (gr.hs) {
            hs[u] = ldp<T, V, LD_NC>(x + idx + gr.mir - gr.hx);
            bs[u] = ldp<T, V, MB>(a.S + idx);
          } else {
            hs[u] = bs[u] = zero_pack<T, V>();
          }
          bu[u] = ldp<T, V, MB>(a.U + idx);
          bd[u] = ldp<T, V, MB>(a.D + idx);
          cc[u] = ldp<T, V, MB>(c + idx);
        }
      }
      T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int k = k0 + u;
        if (k < nz) {
          Pack<T, V> yy;
#pragma unroll
          for (int cl = 0; cl < V; ++cl) {
            T t = x0.a[cl];
            t = fma(be[u].a[cl], nbr_e<T, V>(gr, hm[u], hx1[u], cl), t);
            t = fma(bw[u].a[cl], nbr_w<T, V>(gr, hm[u], hx1[u], cl), t);
            t = fma(bn[u].a[cl], hn[u].a[cl], t);
            t = fma(bs[u].a[cl], hs[u].a[cl], t);
            t = fma(bu[u].a[cl], xp[u].a[cl], t);
            t = fma(bd[u].a[cl], xm.a[cl], t);
            yy.a[cl] = t;
            a0 = fma(cc[u].a[cl], t, a0);
            if (MODE == 1) {
              a1 = fma(t, t, a1);
              a2 = fma(cc[u].a[cl], cc[u].a[cl], a2);
            }
          }
          stp<T, V, SY>(y + (int64_t)k * ncol + q0, yy);
          xm = x0;
          x0 = xp[u];
        }
      }
      acc0.add(a0);
      if (MODE == 1) {
        acc1.add(a1);
        acc2.add(a2);
      }
    }
  }
  const bool f32 = sizeof(T) == 4 && ctl->dot32;
  if (MODE == 0) {
    double vv[1] = {acc0.total(f32)}, o[1];
    if (grid_reduce<1>(vv, red, o, f32)) fin_alpha(ctl, o[0]);
  } else {
    double vv[3] = {acc0.total(f32), acc1.total(f32), acc2.total(f32)}, o[3];
    if (grid_reduce<3>(vv, red, o, f32)) {
      fin_snorm(ctl, o[2]);
      if (ctl->state == ST_RUNNING) fin_omega(ctl, o[0], o[1]);
    }
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

// blocks of kBS threads for the interleaved both-colour kernels with V columns per thread
inline int64_t rb_blocks(const Grid& g, int V) { return 2 * ((g.ncol / 2 / V + kBS - 1) / kBS); }

template <typename T>
cudaError_t launch_sor_first(const Grid& g, const Bands<T>& a, const Vecs<T>& w, T* z1, double omega, int mode,
                             Ctl* ctl, Red red, const Launch& L) {
  return with_sor<T, 2>(L.vsor[sor_prec<T>()][2], [&](auto vc, auto uc, auto bc, auto hc) {
    constexpr int V = decltype(vc)::value, U = decltype(uc)::value, B = decltype(bc)::value;
    constexpr bool H = decltype(hc)::value;
    if ((g.nx / 2) % V) return cudaErrorInvalidValue;
    const int64_t wb = rb_blocks(g, V);
    if (mode == 0)
      k_sor_first<T, 0, V, U, B, H><<<grid_for((const void*)k_sor_first<T, 0, V, U, B, H>, kBS, L, wb), kBS, 0,
                                      L.stream>>>(g, a, w, z1, omega, ctl, red);
    else
      k_sor_first<T, 1, V, U, B, H><<<grid_for((const void*)k_sor_first<T, 1, V, U, B, H>, kBS, L, wb), kBS, 0,
                                      L.stream>>>(g, a, w, z1, omega, ctl, red);
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_sor_pass(const Grid& g, const Bands<T>& a, const T* rc, const T* znbr, const T* zold, T* zout,
                            int colour, int nbr, double omega, const Ctl* ctl, const Launch& L) {
  return with_sor<T, 0>(L.vsor[sor_prec<T>()][0], [&](auto vc, auto uc, auto bc, auto hc) {
    constexpr int V = decltype(vc)::value, U = decltype(uc)::value, B = decltype(bc)::value;
    constexpr bool H = decltype(hc)::value;
    if ((g.nx / 2) % V) return cudaErrorInvalidValue;
    const int64_t wb = (g.ncol / 2 / V + kBS - 1) / kBS;
    k_sor_pass<T, V, U, B, H><<<grid_for((const void*)k_sor_pass<T, V, U, B, H>, kBS, L, wb), kBS, 0, L.stream>>>(
        g, a, rc, znbr, zold, zout, colour, nbr, omega, ctl);
    return cudaGetLastError();
  });
}

template <typename T>
cudaError_t launch_mv_rb(const Grid& g, const Bands<T>& a, const Vecs<T>& w, int mode, Ctl* ctl, Red red,
                         const Launch& L) {
  return with_sor<T, 1>(L.vsor[sor_prec<T>()][1], [&](auto vc, auto uc, auto bc, auto hc) {
    constexpr int V = decltype(vc)::value, U = decltype(uc)::value, B = decltype(bc)::value;
    constexpr bool H = decltype(hc)::value;
    if ((g.nx / 2) % V) return cudaErrorInvalidValue;
    const int64_t wb = rb_blocks(g, V);
    if (mode == 0)
      k_mv_rb<T, 0, V, U, B, H><<<grid_for((const void*)k_mv_rb<T, 0, V, U, B, H>, kBS, L, wb), kBS, 0, L.stream>>>(
          g, a, w, ctl, red);
    else
      k_mv_rb<T, 1, V, U, B, H><<<grid_for((const void*)k_mv_rb<T, 1, V, U, B, H>, kBS, L, wb), kBS, 0, L.stream>>>(
          g, a, w, ctl, red);
    return cudaGetLastError();
  });
}

template <typename T>
void warm_sor(const Launch& L) {
  grid_for((const void*)k_rb_copy<T, true>, kBS, L, 1);
  grid_for((const void*)k_rb_copy<T, false>, kBS, L, 1);
  for (int id = 0; id < SorVar<T>::NK[0]; ++id)
    with_sor<T, 0>(id, [&](auto vc, auto uc, auto bc, auto hc) {
      grid_for((const void*)k_sor_pass<T, decltype(vc)::value, decltype(uc)::value, decltype(bc)::value,
                                       decltype(hc)::value>,
               kBS, L, 1);
      return cudaSuccess;
    });
  for (int id = 0; id < SorVar<T>::NK[1]; ++id)
    with_sor<T, 1>(id, [&](auto vc, auto uc, auto bc, auto hc) {
      constexpr int V = decltype(vc)::value, U = decltype(uc)::value, B = decltype(bc)::value;
      constexpr bool H = decltype(hc)::value;
      grid_for((const void*)k_mv_rb<T, 0, V, U, B, H>, kBS, L, 1);
      grid_for((const void*)k_mv_rb<T, 1, V, U, B, H>, kBS, L, 1);
      return cudaSuccess;
    });
  for (int id = 0; id < SorVar<T>::NK[2]; ++id)
    with_sor<T, 2>(id, [&](auto vc, auto uc, auto bc, auto hc) {
      constexpr int V = decltype(vc)::value, U = decltype(uc)::value, B = decltype(bc)::value;
      constexpr bool H = decltype(hc)::value;
      grid_for((const void*)k_sor_first<T, 0, V, U, B, H>, kBS, L, 1);
      grid_for((const void*)k_sor_first<T, 1, V, U, B, H>, kBS, L, 1);
      return cudaSuccess;
    });
}

int sor_num_variants(int prec, int kind) {
  if (kind < 0 || kind > 2) return 0;
  return prec == 0 ? SorVar<float>::NK[kind] : SorVar<double>::NK[kind];
}

void sor_variant_shape(int prec, int kind, int id, int* vec, int* depth, int* minb) {
  *vec = prec == 0 ? SorVar<float>::v[kind][id] : SorVar<double>::v[kind][id];
  *depth = prec == 0 ? SorVar<float>::u[kind][id] : SorVar<double>::u[kind][id];
  *minb = prec == 0 ? SorVar<float>::b[kind][id] : SorVar<double>::b[kind][id];
}

bool sor_variant_ok(int prec, int kind, int id, int nx) {
  if (id < 0 || id >= sor_num_variants(prec, kind) || nx % 2) return false;
  int v = 1, u = 1, b = 1;
  sor_variant_shape(prec, kind, id, &v, &u, &b);
  return (nx / 2) % v == 0;
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
