// hz_batched.cu -- many independent systems (uneven grids, or several
// right-hand sides of one operator) solved in one persistent, cooperative
// launch: the whole mixed-precision solve, refinement loop included.
//
// Every phase runs over one global list of work items; an item is one
// block-iteration (kBS column groups) of one system, so systems of different
// sizes are load-balanced by items.  The refinement loop (the FP64 true
// residual of Sec. 3 fused with the update x <- x + d and the FP32 scaling of
// the next right-hand side; then per system the tests on tol, the step limit
// and stagnation) alternates with the inner FP32 BiCGStab (the same iteration
// and control steps as the single-system kernels).  Each system keeps its own
// scalars, state and refinement state in its control block; systems that are
// done are masked out of every phase.  No host round trip is needed, so the
// launch can be captured in a CUDA graph.
// Phases are separated by a grid barrier whose wait is bounded (%globaltimer):
// a block that waits longer than the limit sets an error flag, every block
// leaves, and the host reports HZ_ERR_TIMEOUT -- no spin is unbounded.
//
// Per-system dot products: each block sums its items' partials per system in
// a fixed order, stores them in its own slot, and after the barrier the first
// warp of block b (b < number of systems) adds system b's slots in a fixed
// order and its lane 0 runs the control step -- deterministic for a given
// launch shape.
#include <cstring>
#include <algorithm>
#include <mutex>
#include <vector>

#include "hz_krylov.cuh"

namespace hz {

struct BatchArgs {
  const SysDesc* sys;
  int nsys;
  int64_t nitems;
  int64_t nlitems;     // level items (stencil and update phases)
  double* part;        // [gridDim.x][kMaxSys][4] partial sums
  unsigned* bar;       // [0] arrivals, [1] generation
  int* err;            // bit 0: a barrier wait timed out
  long long timeout_ns;
  int leave_block;     // test hook: this block leaves after its first barrier (-1: none)
  int max_loops;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier with a bounded wait.  Returns false (in every thread of the
// block) once any block has given up; the caller then leaves the kernel.
__device__ bool grid_sync(const BatchArgs& A) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* genp = A.bar + 1;
    volatile int* errp = A.err;
    const unsigned gen = *genp;
    __threadfence();
    const unsigned arrived = atomicAdd(A.bar, 1u);
    if (arrived == gridDim.x - 1) {
      A.bar[0] = 0u;  // reset before the release: nobody passes until gen moves
      __threadfence();
      atomicAdd(A.bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*genp == gen) {
        if (*errp) break;
        if (global_ns() - t0 > (unsigned long long)A.timeout_ns) {
          atomicOr(A.err, 1);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_ok = (*errp == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// per-system control values a phase needs, read through L2 (other blocks write them)
struct SysCtl {
  int state, fresh, rsel, r0sel, xzero;
  float alpha, beta, omega;
};

__device__ void load_ctl(const BatchArgs& A, SysCtl* sc) {
  for (int s = threadIdx.x; s < A.nsys; s += blockDim.x) {
    const Ctl* c = A.sys[s].ctl;
    sc[s].state = __ldcg(&c->state);
    sc[s].fresh = __ldcg(&c->fresh);
    sc[s].rsel = __ldcg(&c->rsel);
    sc[s].r0sel = __ldcg(&c->r0sel);
    sc[s].xzero = __ldcg(&c->xzero);
    sc[s].alpha = (float)__ldcg(&c->alpha);
    sc[s].beta = (float)__ldcg(&c->beta);
    sc[s].omega = (float)__ldcg(&c->omega);
  }
  __syncthreads();
}

// the system of a work item: the last system whose first item is <= item
// (first items in shared memory, ascending, the first one 0)
__device__ __forceinline__ int sys_of(const int64_t* item0, int nsys, int64_t item) {
  int lo = 0, hi = nsys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (item >= item0[mid])
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// block sum of ND values per thread in fixed order; thread 0 adds them to acc
template <int ND>
__device__ __forceinline__ void block_add(double (&v)[ND], double* acc) {
  __shared__ double sm[ND][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    double x = v[d];
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sm[d][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      double x = 0.0;
      for (int w = 0; w < nw; ++w) x += sm[d][w];
      acc[d] += x;
    }
  }
  __syncthreads();
}

// Fixed-order sums of system s's slots d0 .. d0+ND-1 over all blocks, taken by
// one whole warp: lane l adds the slots of blocks l, l+32, l+64, ... in that
// order, then an xor butterfly combines the lanes.  Addition is commutative,
// so every stage leaves the same bits in both partners and every lane ends
// with the same totals; the order depends on the grid size only.
template <int ND>
__device__ __forceinline__ void slots_sum(const BatchArgs& A, int s, int d0, double (&out)[ND]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 0; d < ND; ++d) out[d] = 0.0;
#pragma unroll 4
  for (int b = lane; b < (int)gridDim.x; b += 32) {
    const double* p = A.part + ((size_t)b * kMaxSys + s) * 4 + d0;
#pragma unroll
    for (int d = 0; d < ND; ++d) out[d] += __ldcg(p + d);
  }
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int o = 16; o; o >>= 1) out[d] += __shfl_xor_sync(0xffffffffu, out[d], o);
}

// restart of one column inside the persistent kernel: x of neighbouring
// columns was written by other blocks, so it is read through L2
__device__ double restart_column_cg(const Grid& g, int64_t col, const Bands<float>& a, const Vecs<float>& w,
                                    bool xzero) {
  const int i = (int)(col % g.nx), j = (int)(col / g.nx);
  const int64_t ie = (i == g.nx - 1) ? -(int64_t)(g.nx - 1) : 1;
  const int64_t iw = (i == 0) ? (int64_t)(g.nx - 1) : -1;
  float cacc = 0.f;
  for (int k = 0; k < g.nz; ++k) {
    const int64_t idx = (int64_t)k * g.ncol + col;
    float rk = __ldcg(w.rhs + idx);
    if (!xzero) {
      float y = __ldcg(w.x + idx);
      y = fmaf(a.E[idx], __ldcg(w.x + idx + ie), y);
      y = fmaf(a.W[idx], __ldcg(w.x + idx + iw), y);
      if (j + 1 < g.ny) y = fmaf(a.N[idx], __ldcg(w.x + idx + g.nx), y);
      if (j > 0) y = fmaf(a.S[idx], __ldcg(w.x + idx - g.nx), y);
      if (k + 1 < g.nz) y = fmaf(a.U[idx], __ldcg(w.x + idx + g.ncol), y);
      if (k > 0) y = fmaf(a.D[idx], __ldcg(w.x + idx - g.ncol), y);
      rk -= y;
    }
    w.r[idx] = rk;
    w.r0[idx] = rk;
    cacc = fmaf(rk, rk, cacc);
  }
  SrcCopy<float, 1, LD_CG> src{w.r, w.p};
  thomas_vec<float, 1, 4>(g, col, a.m, a.l, a.cp, w.ph, src);
  return (double)cacc;
}

// The FP64 true residual of one column at levels [k0, k1) (Sec. 3: r = b - A x
// with the unscaled bands) for x = xin + delta (xin absent when hasx is false,
// delta when used is false); writes x to xout (if given), the next inner
// right-hand side rhs = fp32(r / A_C), and adds ||r||^2, ||b||^2, ||rhs||^2.
// x and delta were written by other blocks of this launch: read through L2.
// xin and xout are different buffers, so level chunks of a column may run in
// any order.
__device__ void resid_column(const SysDesc& d, int64_t col, int k0, int k1, bool hasx, const double* xin, bool used,
                             double* xout, double& rr, double& bb, double& hh) {
  const Grid& g = d.g;
  const int64_t n = g.n, ncol = g.ncol;
  const int i = (int)(col % g.nx), j = (int)(col / g.nx);
  const int64_t ie = (i == g.nx - 1) ? -(int64_t)(g.nx - 1) : 1;
  const int64_t iw = (i == 0) ? (int64_t)(g.nx - 1) : -1;
  const bool hn = j + 1 < g.ny, hs = j > 0;
  const bool any = hasx || used;
  auto X = [&](int64_t q) -> double {
    double v = hasx ? __ldcg(xin + q) : 0.0;
    if (used) v += (double)__ldcg(d.w.x + q);
    return v;
  };
  double xm = 0.0, xc = 0.0, xp = 0.0;
  if (any) {
    const int64_t c0 = (int64_t)k0 * ncol + col;
    xm = k0 > 0 ? X(c0 - ncol) : 0.0;
    xc = X(c0);
    xp = k0 + 1 < g.nz ? X(c0 + ncol) : 0.0;
  }
  double crr = 0.0, cbb = 0.0, chh = 0.0;
  for (int k = k0; k < k1; ++k) {
    const int64_t idx = (int64_t)k * ncol + col;
    const double C = __ldg(d.A7 + idx);
    double ax = 0.0;
    if (any) {
      ax = C * xc;
      ax = fma(__ldg(d.A7 + n + idx), X(idx + ie), ax);
      ax = fma(__ldg(d.A7 + 2 * n + idx), X(idx + iw), ax);
      if (hn) ax = fma(__ldg(d.A7 + 3 * n + idx), X(idx + g.nx), ax);
      if (hs) ax = fma(__ldg(d.A7 + 4 * n + idx), X(idx - g.nx), ax);
      if (k + 1 < g.nz) ax = fma(__ldg(d.A7 + 5 * n + idx), xp, ax);
      if (k > 0) ax = fma(__ldg(d.A7 + 6 * n + idx), xm, ax);
      if (xout) xout[idx] = xc;
    }
    const double bv = __ldg(d.b + idx);
    const double r = bv - ax;
    const float h = __fmul_rn((float)r, __frcp_rn((float)C));
    d.w.rhs[idx] = h;
    crr = fma(r, r, crr);
    cbb = fma(bv, bv, cbb);
    chh = fma((double)h, (double)h, chh);
    if (any) {
      xm = xc;
      xc = xp;
      xp = (k + 2 < g.nz) ? X(idx + 2 * ncol) : 0.0;
    }
  }
  rr += crr;
  bb += cbb;
  hh += chh;
}

// After a system's residual pass (slot sums rr, bb, hh): its refinement
// decision (the single-system solver's, in device memory) and, when it goes
// on, the control block of its next inner solve.  first: the pass of the
// initial guess.  moved: the pass wrote x into the other buffer.
__device__ void fin_outer(Ctl* c, bool first, bool moved, double rr, double bb, double hh) {
  if (first) {
    c->ob = bb;
    c->outer = 0;
    c->stall = 0;
    c->inner_total = 0;
    c->restart_total = 0;
    c->odone = 0;
    c->ostatus = HZ_OK;
  } else {
    c->inner_total += c->iter;
    c->restart_total += c->restarts;
    c->last_rnorm2 = c->rnorm2;
    c->last_bnorm2 = c->bnorm2;
    c->last_state = c->state;
    c->outer += 1;
    if (moved) {
      c->cur ^= 1;
      c->xz = 0;
    }
  }
  c->res_rr = rr;
  c->res_bb = bb;
  c->res_hh = hh;
  const double R = c->ob > 0.0 ? sqrt(rr / c->ob) : sqrt(rr);
  if (!first) c->Rprev = c->R;
  c->R = R;
  int done = 0, st = HZ_OK;
  if (!isfinite(R) || (!first && c->last_state == ST_NONFINITE)) {
    done = 1;
    st = HZ_ERR_NONFINITE;
  } else if (R <= c->tol) {
    done = 1;
  } else if (c->outer >= c->max_outer) {
    done = 1;
    st = HZ_ERR_NOT_CONVERGED;
  } else if (!first && R > 0.5 * c->Rprev) {  // stagnation: two steps in a row without halving R
    if (++c->stall >= 2) {
      done = 1;
      st = HZ_ERR_NOT_CONVERGED;
    }
  } else if (!first) {
    c->stall = 0;
  }
  if (done) {
    c->odone = 1;
    c->ostatus = st;
    c->state = ST_CONVERGED;  // masked out of the inner phases
    return;
  }
  c->bnorm2 = hh;
  c->stop2 = c->eta * c->eta * hh;
  c->rho = hh;
  c->r0norm2 = hh;
  c->rnorm2 = hh;
  c->snorm2 = 0.0;
  c->alpha = 1.0;
  c->omega = 1.0;
  c->beta = 0.0;
  c->iter = 0;
  c->since = 0;
  c->restarts = 0;
  c->fresh = 1;
  c->rsel = 0;
  c->r0sel = 0;
  c->xzero = 1;
  c->bodies = 0;
  c->state = !isfinite(hh) ? ST_NONFINITE : (hh > 0.0 ? ST_RUNNING : ST_CONVERGED);
}

// Block-shared state of the persistent kernel.  The item loops of the phases
// are separate non-inlined functions over this block, so that each is
// register-allocated on its own instead of as one body holding every phase.
struct BShm {
  BatchArgs A;
  SysCtl sc[kMaxSys];
  double acc[kMaxSys][3];
  int64_t i0[kMaxSys];   // first column item of each system
  int64_t li0[kMaxSys];  // first level item of each system
  int odone[kMaxSys], cur[kMaxSys], xz[kMaxSys], used[kMaxSys];
};

// A level item of system d: `q` its thread's column group, and the chunk's
// levels [k0, k0 + nk) seen as a grid of their own, with off the chunk's first
// index.  The horizontal stencil and the pointwise updates read no other
// level; the residual reads x one level above and below the chunk, which no
// phase writes at the same time.
struct Chunk {
  Grid g;
  int64_t q, off;
  int k0;
};
__device__ __forceinline__ Chunk level_item(const SysDesc& d, int64_t item) {
  const int64_t loc = item - d.litem0;
  const int kc = (int)(loc / d.nitems);
  Chunk c;
  c.q = (loc - (int64_t)kc * d.nitems) * kBS + threadIdx.x;
  const int k0 = kc * d.lchunk;
  const int nk = d.g.nz - k0 < d.lchunk ? d.g.nz - k0 : d.lchunk;
  c.g = d.g;
  c.g.nz = nk;
  c.g.n = (int64_t)nk * d.g.ncol;
  c.off = (int64_t)k0 * d.g.ncol;
  c.k0 = k0;
  return c;
}
__device__ __forceinline__ Bands<float> hbands_at(const Bands<float>& a, int64_t off) {
  Bands<float> b = a;
  b.E += off;
  b.W += off;
  b.N += off;
  b.S += off;
  return b;
}

// ---- phase R items (level items): each active system's FP64 residual (first: of the
// initial guess; else of x + d, the refinement update) ----
template <int V>
__device__ __noinline__ void items_resid(BShm* sh, bool first) {
  const BatchArgs& A = sh->A;
  const int nsys = A.nsys;
  for (int64_t item = blockIdx.x; item < A.nlitems; item += gridDim.x) {
    const int s = sys_of(sh->li0, nsys, item);
    if (sh->odone[s]) continue;
    const SysDesc& d = A.sys[s];
    const Chunk ch = level_item(d, item);
    const int64_t q = ch.q;
    double v[3] = {0.0, 0.0, 0.0};
    if (q < d.g.ncol / V) {
      const double* xin;
      double* xout;
      bool hasx;
      if (first) {  // the initial guess is copied into xa (cur = 0) or x stays zero
        hasx = d.x0 != nullptr;
        xin = d.x0;
        xout = hasx ? d.xa : nullptr;
      } else {
        hasx = !sh->xz[s];
        xin = sh->cur[s] ? d.xb : d.xa;
        xout = (hasx || sh->used[s]) ? (sh->cur[s] ? d.xa : d.xb) : nullptr;
      }
      for (int cc = 0; cc < V; ++cc)
        resid_column(d, q * V + cc, ch.k0, ch.k0 + ch.g.nz, hasx, xin, sh->used[s] != 0, xout, v[0], v[1], v[2]);
    }
    block_add<3>(v, &sh->acc[s][0]);
  }
}

// ---- phase A items: (re)start or p = r + beta (p - omega v); ph = T^-1 p ----
template <int V, int UT>
__device__ __noinline__ void items_pre_p(BShm* sh) {
  const BatchArgs& A = sh->A;
  for (int64_t item = blockIdx.x; item < A.nitems; item += gridDim.x) {
    const int s = sys_of(sh->i0, A.nsys, item);
    const SysCtl c = sh->sc[s];
    if (c.state != ST_RUNNING && c.state != ST_RESTART) continue;
    const SysDesc& d = A.sys[s];
    const int64_t q = (item - d.item0) * kBS + threadIdx.x;
    double v[1] = {0.0};
    if (q < d.g.ncol / V) {
      if (c.state == ST_RESTART) {
        for (int cc = 0; cc < V; ++cc) v[0] += restart_column_cg(d.g, q * V + cc, d.a, d.w, c.xzero != 0);
      } else if (c.fresh) {
        SrcCopy<float, V, LD_CG> src{c.rsel ? d.w.r : d.w.rhs, d.w.p};
        thomas_vec<float, V, UT>(d.g, q * V, d.a.m, d.a.l, d.a.cp, d.w.ph, src);
      } else {
        SrcP<float, V, LD_CG> src{c.rsel ? d.w.r : d.w.rhs, d.w.p, d.w.v, c.beta, c.omega};
        thomas_vec<float, V, UT>(d.g, q * V, d.a.m, d.a.l, d.a.cp, d.w.ph, src);
      }
    }
    if (c.state == ST_RESTART) block_add<1>(v, &sh->acc[s][0]);
  }
}

// ---- phase B items (level items): v = p + H ph, <r0, v> ----
template <int V, int UM>
__device__ __noinline__ void items_mv_v(BShm* sh) {
  const BatchArgs& A = sh->A;
  for (int64_t item = blockIdx.x; item < A.nlitems; item += gridDim.x) {
    const int s = sys_of(sh->li0, A.nsys, item);
    const SysCtl c = sh->sc[s];
    if (c.state != ST_RUNNING && c.state != ST_RESTART) continue;
    const SysDesc& d = A.sys[s];
    const Chunk ch = level_item(d, item);
    double v[1] = {0.0}, dummy = 0.0;
    const bool r0buf = c.r0sel || c.state == ST_RESTART;
    if (ch.q < d.g.ncol / V)
      hmv_vec<float, V, UM, 0, LD_CG>(ch.g, ch.q * V, hbands_at(d.a, ch.off), d.w.p + ch.off, d.w.ph + ch.off,
                                      d.w.v + ch.off, (r0buf ? d.w.r0 : d.w.rhs) + ch.off, v[0], dummy);
    block_add<1>(v, &sh->acc[s][0]);
  }
}

// ---- phase C items: s = r - alpha v, sh = T^-1 s (the test on ||s|| is phase D's) ----
template <int V, int UT>
__device__ __noinline__ void items_pre_s(BShm* sh) {
  const BatchArgs& A = sh->A;
  for (int64_t item = blockIdx.x; item < A.nitems; item += gridDim.x) {
    const int s = sys_of(sh->i0, A.nsys, item);
    const SysCtl c = sh->sc[s];
    if (c.state != ST_RUNNING) continue;
    const SysDesc& d = A.sys[s];
    const int64_t q = (item - d.item0) * kBS + threadIdx.x;
    if (q < d.g.ncol / V) {
      SrcS<float, V, LD_CG, false, false> src{c.rsel ? d.w.r : d.w.rhs, d.w.v, d.w.s, c.alpha, 0.f, {}};
      thomas_vec<float, V, UT>(d.g, q * V, d.a.m, d.a.l, d.a.cp, d.w.sh, src);
    }
  }
}

// ---- phase D items (level items): t = s + H sh, <t, s>, <t, t>, <s, s> ----
template <int V, int UM>
__device__ __noinline__ void items_mv_t(BShm* sh) {
  const BatchArgs& A = sh->A;
  for (int64_t item = blockIdx.x; item < A.nlitems; item += gridDim.x) {
    const int s = sys_of(sh->li0, A.nsys, item);
    const SysCtl c = sh->sc[s];
    if (c.state != ST_RUNNING) continue;
    const SysDesc& d = A.sys[s];
    const Chunk ch = level_item(d, item);
    double v[3] = {0.0, 0.0, 0.0};
    if (ch.q < d.g.ncol / V)
      hmv_vec<float, V, UM, 3, LD_CG>(ch.g, ch.q * V, hbands_at(d.a, ch.off), d.w.s + ch.off, d.w.sh + ch.off,
                                      d.w.t + ch.off, nullptr, v[0], v[1], &v[2]);
    block_add<3>(v, &sh->acc[s][0]);
  }
}

// ---- phase E items (level items): x += alpha ph + omega sh, r = s - omega t, <r0, r>, <r, r> ----
template <int V>
__device__ __noinline__ void items_upd(BShm* sh) {
  const BatchArgs& A = sh->A;
  for (int64_t item = blockIdx.x; item < A.nlitems; item += gridDim.x) {
    const int s = sys_of(sh->li0, A.nsys, item);
    const SysCtl c = sh->sc[s];
    if (c.state != ST_RUNNING && c.state != ST_HALF) continue;
    const SysDesc& d = A.sys[s];
    const Chunk ch = level_item(d, item);
    const int64_t q = ch.q;
    double v[2] = {0.0, 0.0};
    if (q < d.g.ncol / V) {
      const bool half = c.state == ST_HALF;
      const float* r0 = c.r0sel ? d.w.r0 : d.w.rhs;
      DotAcc<float> u0{}, u1{};
      for (int k = 0; k < ch.g.nz; ++k) {
        const int64_t idx = ch.off + (int64_t)k * d.g.ncol + q * V;
        Pack<float, V> xv, pv = ldp<float, V, LD_CG>(d.w.ph + idx);
        if (c.xzero) {
#pragma unroll
          for (int u = 0; u < V; ++u) xv.a[u] = 0.f;
        } else {
          xv = ldp<float, V, LD_CG>(d.w.x + idx);
        }
        if (half) {
#pragma unroll
          for (int u = 0; u < V; ++u) xv.a[u] = fmaf(c.alpha, pv.a[u], xv.a[u]);
        } else {
          const Pack<float, V> shv = ldp<float, V, LD_CG>(d.w.sh + idx), sv = ldp<float, V, LD_CG>(d.w.s + idx),
                               tv = ldp<float, V, LD_CG>(d.w.t + idx), r0v = ldp<float, V, LD_CG>(r0 + idx);
          Pack<float, V> rv;
          float a0 = 0.f, a1 = 0.f;
#pragma unroll
          for (int u = 0; u < V; ++u) {
            xv.a[u] = fmaf(c.omega, shv.a[u], fmaf(c.alpha, pv.a[u], xv.a[u]));
            rv.a[u] = fmaf(-c.omega, tv.a[u], sv.a[u]);
            a0 = fmaf(r0v.a[u], rv.a[u], a0);
            a1 = fmaf(rv.a[u], rv.a[u], a1);
          }
          stp(d.w.r + idx, rv);
          u0.add(a0);
          u1.add(a1);
        }
        stp(d.w.x + idx, xv);
      }
      v[0] = u0.value();
      v[1] = u1.value();
    }
    block_add<2>(v, &sh->acc[s][0]);
  }
}

__device__ __forceinline__ void zero_acc(BShm* sh) {
  for (int s = threadIdx.x; s < sh->A.nsys; s += blockDim.x) sh->acc[s][0] = sh->acc[s][1] = sh->acc[s][2] = 0.0;
  __syncthreads();
}

// this block's partials of slots d0 .. d0+nd-1 (acc columns 0 .. nd-1 hold them)
__device__ __forceinline__ void store_acc(BShm* sh, int d0, int nd) {
  for (int s = threadIdx.x; s < sh->A.nsys; s += blockDim.x)
    for (int d = 0; d < nd; ++d) sh->A.part[((size_t)blockIdx.x * kMaxSys + s) * 4 + d0 + d] = sh->acc[s][d];
  __threadfence();
}

// ---- phase R: the residual items, then each system's refinement decision.
// The refinement steps of all systems are taken together, once every inner
// solve has ended: the phases are latency-bound for small systems, so one
// residual phase for all costs less than one per system (measured: 177 ms
// against 188 ms for 64 systems of 48x36x70 with per-system steps) ----
template <int V>
__device__ bool phase_resid(BShm* sh, bool first) {
  const BatchArgs& A = sh->A;
  const int nsys = A.nsys;
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
    const Ctl* c = A.sys[s].ctl;
    sh->odone[s] = __ldcg(&c->odone);
    sh->cur[s] = __ldcg(&c->cur);
    sh->xz[s] = __ldcg(&c->xz);
    sh->used[s] = !first && __ldcg(&c->xzero) == 0 && __ldcg(&c->state) != ST_NONFINITE;
  }
  __syncthreads();
  zero_acc(sh);
  items_resid<V>(sh, first);
  store_acc(sh, 0, 3);
  if (!grid_sync(A)) return false;
  if ((int)blockIdx.x < nsys && threadIdx.x < 32) {
    const int s = blockIdx.x;
    if (!sh->odone[s]) {
      double t[3];
      slots_sum<3>(A, s, 0, t);
      if (threadIdx.x == 0) {
        const SysDesc& d = A.sys[s];
        const bool moved = !first && (!sh->xz[s] || sh->used[s]);
        fin_outer(d.ctl, first, moved, t[0], t[1], t[2]);
        if (first) {
          d.ctl->cur = 0;
          d.ctl->xz = d.x0 ? 0 : 1;
        }
      }
    }
    if (threadIdx.x == 0) __threadfence();
  }
  return grid_sync(A);
}

template <int V, int UT, int UM>
__global__ void __launch_bounds__(kBS, 4) k_batched(BatchArgs Ain) {
  __shared__ BShm shm;
  BShm* sh = &shm;
  if (threadIdx.x == 0) shm.A = Ain;
  for (int s = threadIdx.x; s < Ain.nsys; s += blockDim.x) {
    shm.i0[s] = Ain.sys[s].item0;
    shm.li0[s] = Ain.sys[s].litem0;
  }
  __syncthreads();
  const BatchArgs& A = shm.A;
  const int nsys = A.nsys;
  SysCtl* sc = shm.sc;

  if (!phase_resid<V>(sh, true)) return;
  if ((int)blockIdx.x == A.leave_block) return;  // test hook: the others must time out, not hang
  for (int loop = 0; loop < A.max_loops; ++loop) {
    load_ctl(A, sc);
    bool any = false;
    for (int s = 0; s < nsys; ++s) any |= (sc[s].state == ST_RUNNING || sc[s].state == ST_RESTART);
    if (!any) {
      // every inner solve is done: the refinement step of each active system
      bool active = false;
      for (int s = 0; s < nsys; ++s) active |= !__ldcg(&A.sys[s].ctl->odone);
      if (!active) break;
      if (!phase_resid<V>(sh, false)) return;
      continue;
    }

    // ---- phase A: (re)start or p = r + beta (p - omega v); ph = T^-1 p ----
    zero_acc(sh);
    items_pre_p<V, UT>(sh);
    store_acc(sh, 0, 1);
    if (!grid_sync(A)) return;

    // ---- phase B: v = p + H ph, <r0, v> ----
    zero_acc(sh);
    items_mv_v<V, UM>(sh);
    store_acc(sh, 1, 1);
    if (!grid_sync(A)) return;
    if ((int)blockIdx.x < nsys && threadIdx.x < 32) {
      const int s = blockIdx.x;
      if (sc[s].state == ST_RESTART || sc[s].state == ST_RUNNING) {
        double t[2];
        slots_sum<2>(A, s, 0, t);
        if (threadIdx.x == 0) {
          Ctl* ctl = A.sys[s].ctl;
          if (sc[s].state == ST_RESTART) fin_restart(ctl, t[0]);
          if (ctl->state == ST_RUNNING) fin_alpha(ctl, t[1]);
        }
      }
      if (threadIdx.x == 0) __threadfence();
    }
    if (!grid_sync(A)) return;
    load_ctl(A, sc);

    // ---- phase C: s = r - alpha v, sh = T^-1 s (the test on ||s|| is phase D's) ----
    items_pre_s<V, UT>(sh);
    if (!grid_sync(A)) return;

    // ---- phase D: t = s + H sh, <t, s>, <t, t>, <s, s> -> half-step test, omega ----
    zero_acc(sh);
    items_mv_t<V, UM>(sh);
    store_acc(sh, 0, 3);
    if (!grid_sync(A)) return;
    if ((int)blockIdx.x < nsys && threadIdx.x < 32) {
      const int s = blockIdx.x;
      if (sc[s].state == ST_RUNNING) {
        double t[3];
        slots_sum<3>(A, s, 0, t);
        if (threadIdx.x == 0) {
          Ctl* ctl = A.sys[s].ctl;
          fin_snorm(ctl, t[2]);
          if (ctl->state == ST_RUNNING) fin_omega(ctl, t[0], t[1]);
        }
      }
      if (threadIdx.x == 0) __threadfence();
    }
    if (!grid_sync(A)) return;
    load_ctl(A, sc);

    // ---- phase E: x += alpha ph + omega sh, r = s - omega t, <r0, r>, <r, r> ----
    zero_acc(sh);
    items_upd<V>(sh);
    store_acc(sh, 2, 2);
    if (!grid_sync(A)) return;
    if ((int)blockIdx.x < nsys && threadIdx.x < 32) {
      const int s = blockIdx.x;
      if (sc[s].state == ST_RUNNING || sc[s].state == ST_HALF) {
        double t[2];
        slots_sum<2>(A, s, 2, t);
        if (threadIdx.x == 0) fin_iteration(A.sys[s].ctl, sc[s].state == ST_HALF, t[0], t[1]);
      }
      if (threadIdx.x == 0) __threadfence();
    }
    if (!grid_sync(A)) return;
  }
  // the result in the caller's buffer: systems whose x ended in the second one
  for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
    shm.cur[s] = __ldcg(&A.sys[s].ctl->cur);
    shm.xz[s] = __ldcg(&A.sys[s].ctl->xz);
  }
  __syncthreads();
  for (int64_t item = blockIdx.x; item < A.nitems; item += gridDim.x) {
    const int s = sys_of(shm.i0, nsys, item);
    const SysDesc& d = A.sys[s];
    const int64_t q = (item - d.item0) * kBS + threadIdx.x;
    if (q >= d.g.ncol / V || (!shm.cur[s] && !shm.xz[s])) continue;
    for (int cc = 0; cc < V; ++cc)
      for (int k = 0; k < d.g.nz; ++k) {
        const int64_t idx = (int64_t)k * d.g.ncol + q * V + cc;
        d.xa[idx] = shm.xz[s] ? 0.0 : __ldcg(d.xb + idx);
      }
  }
}
// ---------------------------------------------------------------------------
struct BatchWs {
  SysDesc* sys = nullptr;
  SysDesc* sys_pin = nullptr;  // pinned host copy (the source of the graph's upload)
  double* part = nullptr;
  unsigned* bar = nullptr;
  int* err = nullptr;
  int part_grid = 0;
  // the captured launch and what it baked in
  cudaGraphExec_t exec = nullptr;
  int g_nsys = 0, g_vec = 0;
  int* g_err_h = nullptr;
  cudaStream_t g_stream = nullptr;
  BatchArgs g_args{};
};

template <int V>
const void* batched_kernel() {
  return V == 4 ? (const void*)k_batched<4, 2, 1> : (const void*)k_batched<1, 4, 4>;
}

// member by member (struct padding is not part of what a launch bakes in)
bool same_sys(const SysDesc& a, const SysDesc& b) {
  const Bands<float>& p = a.a;
  const Bands<float>& q = b.a;
  const Vecs<float>& v = a.w;
  const Vecs<float>& u = b.w;
  return a.g.nx == b.g.nx && a.g.ny == b.g.ny && a.g.nz == b.g.nz && a.item0 == b.item0 && a.nitems == b.nitems &&
         a.litem0 == b.litem0 && a.lchunk == b.lchunk && a.nchunk == b.nchunk &&
         a.ctl == b.ctl && a.A7 == b.A7 && a.invc == b.invc && a.b == b.b && a.x0 == b.x0 && a.xa == b.xa &&
         a.xb == b.xb && p.E == q.E && p.W == q.W && p.N == q.N && p.S == q.S && p.U == q.U && p.D == q.D &&
         p.m == q.m && p.l == q.l && p.cp == q.cp && v.rhs == u.rhs && v.r == u.r && v.r0 == u.r0 && v.p == u.p &&
         v.ph == u.ph && v.v == u.v && v.s == u.s && v.sh == u.sh && v.t == u.t && v.x == u.x;
}
bool same_args(const BatchArgs& a, const BatchArgs& b) {
  return a.sys == b.sys && a.nsys == b.nsys && a.nitems == b.nitems && a.nlitems == b.nlitems && a.part == b.part &&
         a.bar == b.bar &&
         a.err == b.err && a.timeout_ns == b.timeout_ns && a.leave_block == b.leave_block &&
         a.max_loops == b.max_loops;
}

// Launch the persistent kernel cooperatively (or replay its captured graph).
cudaError_t launch_batched(const SysDesc* sys_h, int nsys, int vec, int max_loops, long long timeout_ns,
                           int leave_block, cudaStream_t stream, int* err_h, int sms, bool graph) {
  static BatchWs ws[64];
  static std::mutex mu;  // the per-device workspace is shared by every host thread
  std::lock_guard<std::mutex> lk(mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || nsys > kMaxSys || nsys < 1) return cudaErrorInvalidValue;
  BatchWs& w = ws[dev];
  const void* kern = batched_kernel<4>();
  if (vec != 4) kern = batched_kernel<1>();
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBS, 0)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = per_sm * sms;  // cooperative: every block resident
  if (!w.sys) {
    // allocate into locals and publish only when all exist, so that a failed
    // allocation never leaves a half-built workspace for the next call
    SysDesc* sys = nullptr;
    SysDesc* sys_pin = nullptr;
    unsigned* bar = nullptr;
    int* err = nullptr;
    e = cudaMalloc(&sys, sizeof(SysDesc) * kMaxSys);
    if (e == cudaSuccess) e = cudaMallocHost(&sys_pin, sizeof(SysDesc) * kMaxSys);
    if (e == cudaSuccess) e = cudaMalloc(&bar, sizeof(unsigned) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e != cudaSuccess) {
      if (sys) cudaFree(sys);
      if (sys_pin) cudaFreeHost(sys_pin);
      if (bar) cudaFree(bar);
      return e;
    }
    w.sys = sys;
    w.sys_pin = sys_pin;
    w.bar = bar;
    w.err = err;
  }
  if (w.part_grid < grid) {
    double* part = nullptr;
    if ((e = cudaMalloc(&part, sizeof(double) * (size_t)grid * kMaxSys * 4)) != cudaSuccess) return e;
    if (w.part) cudaFree(w.part);
    w.part = part;
    w.part_grid = grid;
    if (w.exec) cudaGraphExecDestroy(w.exec), w.exec = nullptr;  // it baked the old buffer in
  }
  int64_t nitems = 0;
  for (int s = 0; s < nsys; ++s) nitems = sys_h[s].item0 + sys_h[s].nitems;
  // Level chunks for the stencil and update phases: a batch with fewer column
  // items than two per block splits each system's levels (chunks of at least 8
  // levels), so that those phases are not one thread's march down every level.
  std::vector<SysDesc> loc(sys_h, sys_h + nsys);
  const int64_t target = nitems >= 2 * (int64_t)grid ? 1 : (2 * (int64_t)grid + nitems - 1) / nitems;
  int64_t nlitems = 0;
  for (auto& d : loc) {
    const int64_t nch = std::min<int64_t>(target, std::max(1, d.g.nz / 8));
    d.lchunk = (int)((d.g.nz + nch - 1) / nch);
    d.nchunk = (d.g.nz + d.lchunk - 1) / d.lchunk;
    d.litem0 = nlitems;
    nlitems += d.nitems * d.nchunk;
  }
  BatchArgs args{w.sys, nsys, nitems, nlitems, w.part, w.bar, w.err, timeout_ns, leave_block, max_loops};
  // the launch's inputs, as a graph would bake them in
  bool same = w.exec && w.g_nsys == nsys && w.g_vec == vec && w.g_err_h == err_h && w.g_stream == stream &&
              same_args(w.g_args, args);
  for (int s = 0; same && s < nsys; ++s) same = same_sys(w.sys_pin[s], loc[s]);
  if (graph && same) return cudaGraphLaunch(w.exec, stream);
  memcpy(w.sys_pin, loc.data(), sizeof(SysDesc) * nsys);
  auto enqueue = [&]() -> cudaError_t {
    cudaError_t r;
    if ((r = cudaMemcpyAsync(w.sys, w.sys_pin, sizeof(SysDesc) * nsys, cudaMemcpyHostToDevice, stream)) != cudaSuccess)
      return r;
    if ((r = cudaMemsetAsync(w.bar, 0, sizeof(unsigned) * 2, stream)) != cudaSuccess) return r;
    if ((r = cudaMemsetAsync(w.err, 0, sizeof(int), stream)) != cudaSuccess) return r;
    void* kargs[] = {&args};
    if ((r = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kBS), kargs, 0, stream)) != cudaSuccess) return r;
    return cudaMemcpyAsync(err_h, w.err, sizeof(int), cudaMemcpyDeviceToHost, stream);
  };
  if (graph) {
    if (w.exec) cudaGraphExecDestroy(w.exec), w.exec = nullptr;
    cudaGraph_t gr = nullptr;
    cudaError_t ec = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
    if (ec == cudaSuccess) {
      const cudaError_t eq = enqueue();
      ec = cudaStreamEndCapture(stream, &gr);
      if (eq == cudaSuccess && ec == cudaSuccess) ec = cudaGraphInstantiate(&w.exec, gr, 0);
      if (gr) cudaGraphDestroy(gr);
      if (eq != cudaSuccess && ec == cudaSuccess) ec = eq;
    }
    if (ec == cudaSuccess) {
      w.g_nsys = nsys;
      w.g_vec = vec;
      w.g_err_h = err_h;
      w.g_stream = stream;
      w.g_args = args;
      return cudaGraphLaunch(w.exec, stream);
    }
    cudaGetLastError();  // not capturable here: launch directly
    if (w.exec) cudaGraphExecDestroy(w.exec), w.exec = nullptr;
  }
  return enqueue();
}

}  // namespace hz
