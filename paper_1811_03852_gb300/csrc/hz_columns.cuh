// hz_columns.cuh -- column-marching building blocks of the inner iteration.
//
// Layout [k][j][i], i fastest.  A thread owns V consecutive columns of one
// latitude row (V = 1, 2 or 4; V must divide nx so that a group never crosses
// a row) and marches k.  Each level of a group is one 4*V-byte (FP32) or
// 8*V-byte (FP64) vector load per array, so a warp reads 32*V contiguous
// elements per array and level.  The march is software-pipelined: the loads
// of U consecutive levels are issued before any of them is used.
#pragma once

#include <type_traits>

#include <cuda_fp16.h>

#include "hz_internal.cuh"

namespace hz {

template <typename T, int V>
struct Pack {
  T a[V];
};

// vector load.  M = LD_PLAIN: coherent (data this thread wrote); LD_NC: read-only
// for the whole launch (non-coherent path); LD_CG: written earlier in the same
// launch by other blocks (L2 only, never a stale L1 line).  LD_NC_EF and
// LD_PLAIN_EF are LD_NC and LD_PLAIN with the L2 evict-first priority: for
// arrays that stream through once per launch, so that L2 keeps what is re-read
// (the parked forward sweep of a Thomas variant, stored evict-last).
enum LoadMode : int { LD_PLAIN = 0, LD_NC = 1, LD_CG = 2, LD_NC_EF = 3, LD_PLAIN_EF = 4 };
// store priority in L2: ST_PLAIN (normal), ST_EF (evict first), ST_EL (evict last)
enum StoreMode : int { ST_PLAIN = 0, ST_EF = 1, ST_EL = 2 };

// L2 cache policies (PTX createpolicy, fraction 1.0: every access of the
// instruction that carries the policy gets the priority)
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// loads with an L2 cache policy, by width: 4, 8 or 16 bytes (FP32 x1/x2/x4,
// FP64 x1/x2).  volatile keeps them in program order: the column kernels issue
// a whole batch of loads before the first use, and a compiler free to sink an
// asm load next to its use would serialise the batch.
template <typename W, bool NC>
__device__ __forceinline__ W ld_hint(const W* p, uint64_t pol) {
  W r;
  if constexpr (std::is_same<W, float>::value) {
    if constexpr (NC)
      asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
    else
      asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol) : "memory");
  } else if constexpr (std::is_same<W, float2>::value) {
    if constexpr (NC)
      asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(r.x), "=f"(r.y) : "l"(p), "l"(pol));
    else
      asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                   : "=f"(r.x), "=f"(r.y)
                   : "l"(p), "l"(pol)
                   : "memory");
  } else if constexpr (std::is_same<W, float4>::value) {
    if constexpr (NC)
      asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
          : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
          : "l"(p), "l"(pol));
    else
      asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                   : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                   : "l"(p), "l"(pol)
                   : "memory");
  } else if constexpr (std::is_same<W, double>::value) {
    if constexpr (NC)
      asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol));
    else
      asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol) : "memory");
  } else {
    static_assert(std::is_same<W, double2>::value, "unsupported load width");
    if constexpr (NC)
      asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(r.x), "=d"(r.y) : "l"(p), "l"(pol));
    else
      asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                   : "=d"(r.x), "=d"(r.y)
                   : "l"(p), "l"(pol)
                   : "memory");
  }
  return r;
}

template <typename W>
__device__ __forceinline__ void st_hint(W* p, const W& v, uint64_t pol) {
  if constexpr (std::is_same<W, float>::value) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
  } else if constexpr (std::is_same<W, float2>::value) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
  } else if constexpr (std::is_same<W, float4>::value) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
  } else if constexpr (std::is_same<W, double>::value) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
  } else {
    static_assert(std::is_same<W, double2>::value, "unsupported store width");
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y), "l"(pol)
                 : "memory");
  }
}

// 16-bit loads with an L2 cache policy (one value)
__device__ __forceinline__ uint16_t ld_hint_u16(const uint16_t* p, uint64_t pol) {
  uint16_t r;
  asm volatile("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(r) : "l"(p), "l"(pol));
  return r;
}

template <typename W, int M>
__device__ __forceinline__ W ldw(const W* p) {
  if constexpr (M == LD_NC)
    return __ldg(p);
  else if constexpr (M == LD_CG)
    return __ldcg(p);
  else if constexpr (M == LD_NC_EF)
    return ld_hint<W, true>(p, l2_evict_first());
  else if constexpr (M == LD_PLAIN_EF)
    return ld_hint<W, false>(p, l2_evict_first());
  else
    return *p;
}

template <typename W, int S>
__device__ __forceinline__ void stw(W* p, const W& v) {
  if constexpr (S == ST_EF)
    st_hint<W>(p, v, l2_evict_first());
  else if constexpr (S == ST_EL)
    st_hint<W>(p, v, l2_evict_last());
  else
    *p = v;
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

template <typename T, int V, int S = ST_PLAIN>
__device__ __forceinline__ void stp(T* p, const Pack<T, V>& v) {
  if constexpr (V == 1) {
    stw<T, S>(p, v.a[0]);
  } else if constexpr (sizeof(T) == 4 && V == 4) {
    stw<float4, S>(reinterpret_cast<float4*>(p), make_float4(v.a[0], v.a[1], v.a[2], v.a[3]));
  } else if constexpr (sizeof(T) == 4 && V == 2) {
    stw<float2, S>(reinterpret_cast<float2*>(p), make_float2(v.a[0], v.a[1]));
  } else if constexpr (sizeof(T) == 8 && V == 2) {
    stw<double2, S>(reinterpret_cast<double2*>(p), make_double2(v.a[0], v.a[1]));
  }
}

// V consecutive 16-bit band values (BF16 or FP16 by HB) widened to FP32; the
// V values are one 2V-byte load (the band arrays are 8-byte aligned at every
// group start)
__device__ __forceinline__ float widen16(uint32_t h, int hb) {
  return hb == HB_BF16 ? __uint_as_float(h << 16) : __half2float(__ushort_as_half((unsigned short)h));
}
template <int HB, int V, int M>
__device__ __forceinline__ Pack<float, V> ld16(const uint16_t* p) {
  static_assert(HB == HB_BF16 || HB == HB_FP16, "16-bit band format");
  constexpr bool EF = (M == LD_NC_EF);
  Pack<float, V> r;
  if constexpr (V == 1) {
    const uint16_t h = EF ? ld_hint_u16(p, l2_evict_first()) : __ldg(reinterpret_cast<const unsigned short*>(p));
    r.a[0] = widen16(h, HB);
  } else if constexpr (V == 2) {
    const uint32_t h = EF ? __float_as_uint(ld_hint<float, true>(reinterpret_cast<const float*>(p), l2_evict_first()))
                          : __ldg(reinterpret_cast<const unsigned int*>(p));
    r.a[0] = widen16(h & 0xFFFFu, HB);
    r.a[1] = widen16(h >> 16, HB);
  } else {
    static_assert(V == 4, "unsupported vector width");
    uint2 h;
    if constexpr (EF) {
      const float2 f = ld_hint<float2, true>(reinterpret_cast<const float2*>(p), l2_evict_first());
      h = make_uint2(__float_as_uint(f.x), __float_as_uint(f.y));
    } else {
      h = __ldg(reinterpret_cast<const uint2*>(p));
    }
    r.a[0] = widen16(h.x & 0xFFFFu, HB);
    r.a[1] = widen16(h.x >> 16, HB);
    r.a[2] = widen16(h.y & 0xFFFFu, HB);
    r.a[3] = widen16(h.y >> 16, HB);
  }
  return r;
}

// horizontal band b (0 E, 1 W, 2 N, 3 S) of V columns at idx: FP32/FP64 or 16-bit by HB
template <typename T, int V, int M, int HB>
__device__ __forceinline__ Pack<T, V> ldband(const Bands<T>& a, int b, int64_t idx) {
  if constexpr (HB == HB_F32) {
    const T* base = b == 0 ? a.E : b == 1 ? a.W : b == 2 ? a.N : a.S;
    return ldp<T, V, M>(base + idx);
  } else {
    static_assert(sizeof(T) == 4, "16-bit bands feed the FP32 kernels");
    return ld16<HB, V, M>(a.h16 + (int64_t)b * a.h16s + idx);
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

// Where a Thomas variant parks the forward sweep y until the back sweep reads
// it: PARK_OUT in the output vector (an L2 hit while the columns in flight fit
// in L2), PARK_SMEM in shared memory, PARK_OUT_L2 in the output vector stored
// with the L2 evict-last priority while every streamed array is loaded and
// stored evict-first, so that the parked values are the last to leave L2.
// PARK_BULK: a different kernel (hz_thomas_bulk.cu): the inputs staged level
// by level into shared memory by bulk copies, y parked in the output vector
// under the L2 evict-last priority.
enum ParkMode : int { PARK_OUT = 0, PARK_SMEM = 1, PARK_OUT_L2 = 2, PARK_BULK = kParkBulk };

// Thomas algorithm on V columns with unit diagonal and pre-computed factors:
// forward y_k = m_k q_k - l_k y_(k-1), back z_k = y_k - c'_k z_(k+1).  The
// input q_k = src.make(values src.load fetched for level k) is the fused
// axpy.  y is parked in out and re-read by the back sweep (PARK_OUT,
// PARK_OUT_L2), or in shared memory ys laid out [level][thread][V] (kBS * V
// values per level; PARK_SMEM), which keeps it off L2 and HBM.
template <typename T, int V, int U, typename Src, int P = PARK_OUT>
__device__ __forceinline__ void thomas_vec(const Grid& g, int64_t c0, const T* __restrict__ m,
                                           const T* __restrict__ l, const T* __restrict__ cp, T* __restrict__ out,
                                           Src& src, T* ys = nullptr) {
  constexpr bool SM = P == PARK_SMEM;
  constexpr int LF = P == PARK_OUT_L2 ? LD_NC_EF : LD_NC;      // factors: streamed once
  constexpr int SY = P == PARK_OUT_L2 ? ST_EL : ST_PLAIN;      // y: re-read by the back sweep
  constexpr int SZ = P == PARK_OUT_L2 ? ST_EF : ST_PLAIN;      // z: written once (drops y's priority)
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
        mm[u] = ldp<T, V, LF>(m + idx);
        ll[u] = ldp<T, V, LF>(l + idx);
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
          stp<T, V, SY>(out + idx, y);
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
        cc[u] = ldp<T, V, LF>(cp + idx);
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
        stp<T, V, SZ>(out + idx, z);
      }
    }
  }
}

// inputs of the Thomas sweeps ------------------------------------------------
// EF: the streamed inputs and outputs carry the L2 evict-first priority (the
// sources of a PARK_OUT_L2 variant; M is then LD_NC)
template <typename T, int V, int M = LD_NC, bool EF = false>
struct SrcP {  // p = r + beta (p - omega v)
  static constexpr int NIN = 3;
  static constexpr int MI = EF ? LD_NC_EF : M, MP = EF ? LD_PLAIN_EF : LD_PLAIN, SO = EF ? ST_EF : ST_PLAIN;
  const T* __restrict__ r;
  T* __restrict__ p;
  const T* __restrict__ v;
  T beta, omega;
  __device__ __forceinline__ void load(int64_t idx, Pack<T, V> (&o)[NIN]) {
    o[0] = ldp<T, V, MI>(r + idx);
    o[1] = ldp<T, V, MP>(p + idx);
    o[2] = ldp<T, V, MI>(v + idx);
  }
  __device__ __forceinline__ Pack<T, V> make(const Pack<T, V> (&o)[NIN], int64_t idx) {
    Pack<T, V> q;
#pragma unroll
    for (int c = 0; c < V; ++c) q.a[c] = fma(beta, fma(-omega, o[2].a[c], o[1].a[c]), o[0].a[c]);
    stp<T, V, SO>(p + idx, q);
    return q;
  }
  __device__ __forceinline__ void flush() {}
};

template <typename T, int V, int M = LD_NC, bool EF = false>
struct SrcCopy {  // q = r, optionally stored to dst
  static constexpr int NIN = 1;
  static constexpr int MI = EF ? LD_NC_EF : M, SO = EF ? ST_EF : ST_PLAIN;
  const T* __restrict__ r;
  T* __restrict__ dst;
  __device__ __forceinline__ void load(int64_t idx, Pack<T, V> (&o)[NIN]) { o[0] = ldp<T, V, MI>(r + idx); }
  __device__ __forceinline__ Pack<T, V> make(const Pack<T, V> (&o)[NIN], int64_t idx) {
    if (dst) stp<T, V, SO>(dst + idx, o[0]);
    return o[0];
  }
  __device__ __forceinline__ void flush() {}
};

// DOT: also accumulate <s, s> (FP32 (or FP64) over one batch, DotAcc across
// batches); the single-system solver leaves it to the stencil kernel, which
// reads s anyway, and keeps the Thomas sweep free of it
template <typename T, int V, int M = LD_NC, bool EF = false, bool DOT = true>
struct SrcS {  // s = r - alpha v
  static constexpr int NIN = 2;
  static constexpr int MI = EF ? LD_NC_EF : M, SO = EF ? ST_EF : ST_PLAIN;
  const T* __restrict__ r;
  const T* __restrict__ v;
  T* __restrict__ s;
  T alpha;
  T part;
  DotAcc<T> acc;
  __device__ __forceinline__ void load(int64_t idx, Pack<T, V> (&o)[NIN]) {
    o[0] = ldp<T, V, MI>(r + idx);
    o[1] = ldp<T, V, MI>(v + idx);
  }
  __device__ __forceinline__ Pack<T, V> make(const Pack<T, V> (&o)[NIN], int64_t idx) {
    Pack<T, V> q;
#pragma unroll
    for (int c = 0; c < V; ++c) {
      q.a[c] = fma(-alpha, o[1].a[c], o[0].a[c]);
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

// y = c + H x on V columns, U levels per batch (H = E, W, N, S bands of Ahat,
// read in FP32/FP64 or, for HB = HB_BF16 / HB_FP16, from their 16-bit copies).
// MODE 0: d0 += <r0, y>.  MODE 1: d0 += <y, c>, d1 += <y, y>.  MODE 2: no dots.
// MODE 3: as MODE 1 and *d2 += <c, c>.  f32: the sums run in FP32 throughout
// (the paper's 32-bit global sums).
// Each batch's dot partial is FP32 (FP64 solver: FP64); the batches of the
// group are summed in a DotAcc and the group's total is added to the FP64
// accumulators.  EF (with M = LD_NC): every array read
// once (c, the bands, r0) and y carry the L2 evict-first priority, so that
// the rows of x, read again as the north and south neighbours of the next
// rows, stay in L2.
template <typename T, int V, int U, int MODE, int M = LD_NC, bool EF = false, int HB = HB_F32>
__device__ __forceinline__ void hmv_vec(const Grid& g, int64_t c0, const Bands<T>& a, const T* __restrict__ cen,
                                        const T* __restrict__ x, T* __restrict__ y, const T* __restrict__ r0,
                                        double& d0, double& d1, double* d2 = nullptr, bool f32 = false) {
  static_assert(!EF || M == LD_NC, "L2 priorities with read-only loads only");
  constexpr bool TWO = MODE == 1 || MODE == 3;  // <y, c> and <y, y>
  constexpr int MS = EF ? LD_NC_EF : M;         // streamed vectors
  constexpr int MB = EF ? LD_NC_EF : LD_NC;     // bands
  constexpr int SY = EF ? ST_EF : ST_PLAIN;
  const GroupNbr nb = group_nbr<V>(g, c0);
  const int64_t ncol = g.ncol, nx = g.nx;
  DotAcc<T> s0{}, s1{}, s2{};
  for (int k0 = 0; k0 < g.nz; k0 += U) {
    Pack<T, V> cc[U], e[U], w[U], nn[U], ss[U], xc[U], xn[U], xs[U], q[U];
    T xw1[U], xe1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + u < g.nz) {
        const int64_t idx = (int64_t)(k0 + u) * ncol + c0;
        cc[u] = ldp<T, V, MS>(cen + idx);
        e[u] = ldband<T, V, MB, HB>(a, 0, idx);
        w[u] = ldband<T, V, MB, HB>(a, 1, idx);
        if constexpr (V > 1) xc[u] = ldp<T, V, M>(x + idx);
        xw1[u] = ldw<T, M>(x + idx + nb.w_off);
        xe1[u] = ldw<T, M>(x + idx + nb.e_off);
        if (nb.hn) {
          nn[u] = ldband<T, V, MB, HB>(a, 2, idx);
          xn[u] = ldp<T, V, M>(x + idx + nx);
        } else {
#pragma unroll
          for (int c = 0; c < V; ++c) nn[u].a[c] = xn[u].a[c] = T(0);
        }
        if (nb.hs) {
          ss[u] = ldband<T, V, MB, HB>(a, 3, idx);
          xs[u] = ldp<T, V, M>(x + idx - nx);
        } else {
#pragma unroll
          for (int c = 0; c < V; ++c) ss[u].a[c] = xs[u].a[c] = T(0);
        }
        if constexpr (MODE == 0) q[u] = ldp<T, V, MS>(r0 + idx);
      }
    }
    T p0 = T(0), p1 = T(0), p2 = T(0);
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
          } else if constexpr (TWO) {
            p0 = fma(t, cc[u].a[c], p0);
            p1 = fma(t, t, p1);
            if constexpr (MODE == 3) p2 = fma(cc[u].a[c], cc[u].a[c], p2);
          }
        }
        stp<T, V, SY>(y + idx, yy);
      }
    }
    if constexpr (MODE != 2) s0.add(p0);
    if constexpr (TWO) s1.add(p1);
    if constexpr (MODE == 3) s2.add(p2);
  }
  if constexpr (MODE != 2) d0 = acc_add(d0, s0.total(f32), f32);
  if constexpr (TWO) d1 = acc_add(d1, s1.total(f32), f32);
  if constexpr (MODE == 3) *d2 = acc_add(*d2, s2.total(f32), f32);
}

}  // namespace hz
