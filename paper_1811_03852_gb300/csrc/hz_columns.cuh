// hz_columns.cuh -- column-marching building blocks of the inner iteration.
//
// Layout [k][j][i], i fastest.  A thread owns V consecutive columns of one
// latitude row (V = 1, 2 or 4; V must divide nx so that a group never crosses
// a row) and marches k.  Each level of a group is one 4*V-byte (FP32) or
// 8*V-byte (FP64) vector load per array, so a warp reads 32*V contiguous
// elements per array and level.  The march is software-pipelined: the loads
// of U consecutive levels are issued before any of them is used.
#pragma once

#include "hz_internal.cuh"

namespace hz {

template <typename T, int V>
struct Pack {
  T a[V];
};

// vector load.  M = LD_PLAIN: coherent (data this thread wrote); LD_NC: read-only
// for the whole launch (non-coherent path); LD_CG: written earlier in the same
// launch by other blocks (L2 only, never a stale L1 line)
enum LoadMode : int { LD_PLAIN = 0, LD_NC = 1, LD_CG = 2 };

template <typename W, int M>
__device__ __forceinline__ W ldw(const W* p) {
  if constexpr (M == LD_NC)
    return __ldg(p);
  else if constexpr (M == LD_CG)
    return __ldcg(p);
  else
    return *p;
}

template <typename T, int V, int M>
__device__ __forceinline__ Pack<T, V> ldp(const T* p) {
  Pack<T, V> r;
  if constexpr (V == 1) {
    r.a[0] = ldw<T, M>(p);
  } else if constexpr (sizeof(T) == 4 && V == 4) {
    const float4 t = ldw<float4, M>(reinterpret_cast<const float4*>(p));
    r.a[0] = t.x;
    r.a[1] = t.y;
    r.a[2] = t.z;
    r.a[3] = t.w;
  } else if constexpr (sizeof(T) == 4 && V == 2) {
    const float2 t = ldw<float2, M>(reinterpret_cast<const float2*>(p));
    r.a[0] = t.x;
    r.a[1] = t.y;
  } else if constexpr (sizeof(T) == 8 && V == 2) {
    const double2 t = ldw<double2, M>(reinterpret_cast<const double2*>(p));
    r.a[0] = t.x;
    r.a[1] = t.y;
  } else {
    static_assert(V == 1, "unsupported vector width");
  }
  return r;
}

template <typename T, int V>
__device__ __forceinline__ void stp(T* p, const Pack<T, V>& v) {
  if constexpr (V == 1) {
    *p = v.a[0];
  } else if constexpr (sizeof(T) == 4 && V == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v.a[0], v.a[1], v.a[2], v.a[3]);
  } else if constexpr (sizeof(T) == 4 && V == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v.a[0], v.a[1]);
  } else if constexpr (sizeof(T) == 8 && V == 2) {
    *reinterpret_cast<double2*>(p) = make_double2(v.a[0], v.a[1]);
  }
}

// neighbours of a group of V columns starting at column c0 (i0 = c0 mod nx):
// w_off / e_off locate the west neighbour of column i0 and the east neighbour
// of column i0+V-1 relative to the group's own index (longitude is periodic).
struct GroupNbr {
  int64_t w_off, e_off;
  bool hn, hs;
};

template <int V>
__device__ __forceinline__ GroupNbr group_nbr(const Grid& g, int64_t c0) {
  const int i0 = (int)(c0 % g.nx);
  const int j = (int)(c0 / g.nx);
  GroupNbr n;
  n.w_off = (i0 == 0) ? (int64_t)(g.nx - 1) : -1;
  n.e_off = (i0 + V == g.nx) ? (int64_t)(V - g.nx) : (int64_t)V;
  n.hn = j + 1 < g.ny;
  n.hs = j > 0;
  return n;
}

// Thomas algorithm on V columns with unit diagonal and pre-computed factors:
// forward y_k = m_k q_k - l_k y_(k-1), back z_k = y_k - c'_k z_(k+1).  The
// input q_k = src.make(values src.load fetched for level k) is the fused
// axpy.  y is parked in out and re-read by the back sweep (an L2 hit while the
// column's footprint stays in L2), or with SM in shared memory ys laid out
// [level][thread][V] (kBS * V values per level), which keeps it off L2 and HBM.
template <typename T, int V, int U, typename Src, bool SM = false>
__device__ __forceinline__ void thomas_vec(const Grid& g, int64_t c0, const T* __restrict__ m,
                                           const T* __restrict__ l, const T* __restrict__ cp, T* __restrict__ out,
                                           Src& src, T* ys = nullptr) {
  constexpr int NIN = Src::NIN;
  const int64_t ncol = g.ncol;
  const int nz = g.nz;
  T yprev[V];
#pragma unroll
  for (int c = 0; c < V; ++c) yprev[c] = T(0);
  for (int k0 = 0; k0 < nz; k0 += U) {
    Pack<T, V> v[U][NIN], mm[U], ll[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + c0;
        src.load(idx, v[u]);
        mm[u] = ldp<T, V, LD_NC>(m + idx);
        ll[u] = ldp<T, V, LD_NC>(l + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + c0;
        const Pack<T, V> q = src.make(v[u], idx);
        Pack<T, V> y;
#pragma unroll
        for (int c = 0; c < V; ++c) {
          y.a[c] = fma(mm[u].a[c], q.a[c], -ll[u].a[c] * yprev[c]);
          yprev[c] = y.a[c];
        }
        if constexpr (SM)
          stp(ys + ((int64_t)(k0 + u) * kBS + threadIdx.x) * V, y);
        else
          stp(out + idx, y);
      }
    }
    src.flush();
  }
  T zn[V];
#pragma unroll
  for (int c = 0; c < V; ++c) zn[c] = T(0);
  for (int k0 = nz - 1; k0 >= 0; k0 -= U) {
    Pack<T, V> yy[U], cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 - u >= 0) {
        const int64_t idx = (int64_t)(k0 - u) * ncol + c0;
        if constexpr (SM)
          yy[u] = ldp<T, V, LD_PLAIN>(ys + ((int64_t)(k0 - u) * kBS + threadIdx.x) * V);
        else
          yy[u] = ldp<T, V, LD_PLAIN>(out + idx);  // written by this thread above: coherent load
        cc[u] = ldp<T, V, LD_NC>(cp + idx);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 - u >= 0) {
        const int64_t idx = (int64_t)(k0 - u) * ncol + c0;
        Pack<T, V> z;
#pragma unroll
        for (int c = 0; c < V; ++c) {
          z.a[c] = fma(-cc[u].a[c], zn[c], yy[u].a[c]);
          zn[c] = z.a[c];
        }
        stp(out + idx, z);
      }
    }
  }
}

// inputs of the Thomas sweeps ------------------------------------------------
template <typename T, int V, int M = LD_NC>
struct SrcP {  // p = r + beta (p - omega v)
  static constexpr int NIN = 3;
  const T* __restrict__ r;
  T* __restrict__ p;
  const T* __restrict__ v;
  T beta, omega;
  __device__ __forceinline__ void load(int64_t idx, Pack<T, V> (&o)[NIN]) {
    o[0] = ldp<T, V, M>(r + idx);
    o[1] = ldp<T, V, LD_PLAIN>(p + idx);
    o[2] = ldp<T, V, M>(v + idx);
  }
  __device__ __forceinline__ Pack<T, V> make(const Pack<T, V> (&o)[NIN], int64_t idx) {
    Pack<T, V> q;
#pragma unroll
    for (int c = 0; c < V; ++c) q.a[c] = fma(beta, fma(-omega, o[2].a[c], o[1].a[c]), o[0].a[c]);
    stp(p + idx, q);
    return q;
  }
  __device__ __forceinline__ void flush() {}
};

template <typename T, int V, int M = LD_NC>
struct SrcCopy {  // q = r, optionally stored to dst
  static constexpr int NIN = 1;
  const T* __restrict__ r;
  T* __restrict__ dst;
  __device__ __forceinline__ void load(int64_t idx, Pack<T, V> (&o)[NIN]) { o[0] = ldp<T, V, M>(r + idx); }
  __device__ __forceinline__ Pack<T, V> make(const Pack<T, V> (&o)[NIN], int64_t idx) {
    if (dst) stp(dst + idx, o[0]);
    return o[0];
  }
  __device__ __forceinline__ void flush() {}
};

template <typename T, int V, int M = LD_NC>
struct SrcS {  // s = r - alpha v, with <s, s>: FP32 (or FP64) over one batch, FP64 across batches
  static constexpr int NIN = 2;
  const T* __restrict__ r;
  const T* __restrict__ v;
  T* __restrict__ s;
  T alpha;
  T part;
  double acc;
  __device__ __forceinline__ void load(int64_t idx, Pack<T, V> (&o)[NIN]) {
    o[0] = ldp<T, V, M>(r + idx);
    o[1] = ldp<T, V, M>(v + idx);
  }
  __device__ __forceinline__ Pack<T, V> make(const Pack<T, V> (&o)[NIN], int64_t idx) {
    Pack<T, V> q;
#pragma unroll
    for (int c = 0; c < V; ++c) {
      q.a[c] = fma(-alpha, o[1].a[c], o[0].a[c]);
      part = fma(q.a[c], q.a[c], part);
    }
    stp(s + idx, q);
    return q;
  }
  __device__ __forceinline__ void flush() {
    acc += (double)part;
    part = T(0);
  }
};

// y = c + H x on V columns, U levels per batch (H = E, W, N, S bands of Ahat).
// MODE 0: d0 += <r0, y>.  MODE 1: d0 += <y, c>, d1 += <y, y>.  MODE 2: no dots.
// Each batch's dot partial is FP32 (FP64 solver: FP64) and is added to the
// FP64 accumulators once per batch.
template <typename T, int V, int U, int MODE, int M = LD_NC>
__device__ __forceinline__ void hmv_vec(const Grid& g, int64_t c0, const Bands<T>& a, const T* __restrict__ cen,
                                        const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ r0,
                                        double& d0, double& d1) {
  const GroupNbr nb = group_nbr<V>(g, c0);
  const int64_t ncol = g.ncol, nx = g.nx;
  for (int k0 = 0; k0 < g.nz; k0 += U) {
    Pack<T, V> cc[U], e[U], w[U], nn[U], ss[U], xc[U], xn[U], xs[U], q[U];
    T xw1[U], xe1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < g.nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + c0;
        cc[u] = ldp<T, V, M>(cen + idx);
        e[u] = ldp<T, V, LD_NC>(a.E + idx);
        w[u] = ldp<T, V, LD_NC>(a.W + idx);
        if constexpr (V > 1) xc[u] = ldp<T, V, M>(x + idx);
        xw1[u] = ldw<T, M>(x + idx + nb.w_off);
        xe1[u] = ldw<T, M>(x + idx + nb.e_off);
        if (nb.hn) {
          nn[u] = ldp<T, V, LD_NC>(a.N + idx);
          xn[u] = ldp<T, V, M>(x + idx + nx);
        } else {
#pragma unroll
          for (int c = 0; c < V; ++c) nn[u].a[c] = xn[u].a[c] = T(0);
        }
        if (nb.hs) {
          ss[u] = ldp<T, V, LD_NC>(a.S + idx);
          xs[u] = ldp<T, V, M>(x + idx - nx);
        } else {
#pragma unroll
          for (int c = 0; c < V; ++c) ss[u].a[c] = xs[u].a[c] = T(0);
        }
        if constexpr (MODE == 0) q[u] = ldp<T, V, M>(r0 + idx);
      }
    }
    T p0 = T(0), p1 = T(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < g.nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + c0;
        Pack<T, V> yy;
#pragma unroll
        for (int c = 0; c < V; ++c) {
          const T xe = (c + 1 < V) ? xc[u].a[(c + 1) % V] : xe1[u];
          const T xw = (c > 0) ? xc[u].a[(c + V - 1) % V] : xw1[u];
          T t = fma(e[u].a[c], xe, cc[u].a[c]);
          t = fma(w[u].a[c], xw, t);
          t = fma(nn[u].a[c], xn[u].a[c], t);
          t = fma(ss[u].a[c], xs[u].a[c], t);
          yy.a[c] = t;
          if constexpr (MODE == 0) {
            p0 = fma(q[u].a[c], t, p0);
          } else if constexpr (MODE == 1) {
            p0 = fma(t, cc[u].a[c], p0);
            p1 = fma(t, t, p1);
          }
        }
        stp(y + idx, yy);
      }
    }
    d0 += (double)p0;
    d1 += (double)p1;
  }
}

}  // namespace hz
