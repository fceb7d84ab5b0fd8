// hz_fgmres.cu -- kernels of the flexible GMRES(m) inner solver (FP32 vectors,
// FP64 scalars).
//
// FGMRES (Saad 1993) is right-preconditioned GMRES that stores the
// preconditioned directions z_j = M_j(v_j), so M may change from step to step
// (the learned stage is not a fixed linear operator).  Arnoldi uses classical
// Gram-Schmidt applied twice (CGS2): h = V^T w, w -= V h, twice.  The small
// Hessenberg least-squares problem is solved with Givens rotations in FP64 by
// one thread.  Dots are deterministic: per-block partials in fixed slots,
// summed in slot order by one block.
#include "hz_internal.cuh"

namespace hz {

constexpr int kChunk = 8;  // vectors per multi-dot pass

// partial dots of w with V[q0 .. q0+nq) (nq <= kChunk); slot [block][q0+q]
__global__ void __launch_bounds__(256) k_mdot(int64_t n, float* const* V, int q0, int nq, const float* __restrict__ w,
                                              double* __restrict__ part, int pstride) {
  // FP32 partials over at most 64 elements per thread, FP64 beyond
  double acc[kChunk];
  float pf[kChunk];
#pragma unroll
  for (int q = 0; q < kChunk; ++q) acc[q] = 0.0, pf[q] = 0.f;
  const float* vq[kChunk];
#pragma unroll
  for (int q = 0; q < kChunk; ++q) vq[q] = q < nq ? V[q0 + q] : nullptr;
  int cnt = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float we = w[e];
#pragma unroll
    for (int q = 0; q < kChunk; ++q)
      if (q < nq) pf[q] = fmaf(vq[q][e], we, pf[q]);
    if (++cnt == 64) {
#pragma unroll
      for (int q = 0; q < kChunk; ++q) acc[q] += (double)pf[q], pf[q] = 0.f;
      cnt = 0;
    }
  }
#pragma unroll
  for (int q = 0; q < kChunk; ++q) acc[q] += (double)pf[q];
  __shared__ double sm[kChunk][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kChunk; ++q) {
    double x = acc[q];
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sm[q][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double x = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) x += sm[threadIdx.x][wi];
    part[(size_t)blockIdx.x * pstride + q0 + threadIdx.x] = x;
  }
}

// w -= sum_q c[q] V[q] for q < nv (coefficients in device memory);
// optionally also the partial ||w||^2 in slot [block][0]
__global__ void __launch_bounds__(256) k_mupdate(int64_t n, float* const* V, int nv, const double* __restrict__ c,
                                                 float* __restrict__ w, double* __restrict__ part, int pstride,
                                                 int want_norm) {
  __shared__ float cs[kMaxFgm + 1];
  for (int q = threadIdx.x; q < nv; q += blockDim.x) cs[q] = (float)c[q];
  __syncthreads();
  double nrm = 0.0;
  float pn = 0.f;
  int cnt = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    float we = w[e];
    for (int q = 0; q < nv; ++q) we = fmaf(-cs[q], V[q][e], we);
    w[e] = we;
    pn = fmaf(we, we, pn);
    if (++cnt == 64) {
      nrm += (double)pn;
      pn = 0.f;
      cnt = 0;
    }
  }
  nrm += (double)pn;
  if (!want_norm) return;
  __shared__ double sm[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) sm[warp] = nrm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) x += sm[wi];
    part[(size_t)blockIdx.x * pstride] = x;
  }
}

// out[q] = sum over blocks of part[b][q] (slot order), q < nq; one block
__global__ void k_psum(const double* __restrict__ part, int pstride, int nblocks, int nq, double* __restrict__ out) {
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    double x = 0.0;
    for (int b = 0; b < nblocks; ++b) x += part[(size_t)b * pstride + q];
    out[q] = x;
  }
}

// y = a * x (elementwise); a = 1/sqrt(*nrm2) when inv_sqrt, else *a.  x may be
// y (in-place normalisation), so neither is restrict-qualified.
__global__ void __launch_bounds__(256) k_scale(int64_t n, const float* x, float* y, const double* __restrict__ s,
                                               int inv_sqrt) {
  const double sv = *s;
  const float a = (float)(inv_sqrt ? (sv > 0.0 ? 1.0 / sqrt(sv) : 0.0) : sv);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = a * x[e];
}

// Arnoldi bookkeeping of step j (one thread): column j of H = h1 + h2 (CGS2)
// and h(j+1,j) = ||w||; apply the previous rotations, make the new one, update
// g; resid = |g(j+1)|.
__global__ void k_fgm_step(FgmState* st, int j) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m1 = kMaxFgm + 1;
  double* H = st->H + (size_t)j * m1;  // column j
  for (int i = 0; i <= j; ++i) H[i] = st->h1[i] + st->h2[i];
  H[j + 1] = sqrt(st->wn2);
  for (int i = 0; i < j; ++i) {
    const double a = H[i], b = H[i + 1];
    H[i] = st->cs[i] * a + st->sn[i] * b;
    H[i + 1] = -st->sn[i] * a + st->cs[i] * b;
  }
  const double a = H[j], b = H[j + 1];
  const double r = hypot(a, b);
  const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
  st->cs[j] = c;
  st->sn[j] = s;
  H[j] = r;
  H[j + 1] = 0.0;
  st->g[j + 1] = -s * st->g[j];
  st->g[j] = c * st->g[j];
  st->resid = fabs(st->g[j + 1]);
  st->wnorm = sqrt(st->wn2);
}

// back substitution R y = g for the first k columns (one thread)
__global__ void k_fgm_solve(FgmState* st, int k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m1 = kMaxFgm + 1;
  for (int i = k - 1; i >= 0; --i) {
    double s = st->g[i];
    for (int q = i + 1; q < k; ++q) s -= st->H[(size_t)q * m1 + i] * st->y[q];
    const double d = st->H[(size_t)i * m1 + i];
    st->y[i] = d != 0.0 ? s / d : 0.0;
  }
}

// start of a cycle: g = (beta, 0, ...), beta = sqrt(nrm2)
__global__ void k_fgm_start(FgmState* st, const double* nrm2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st->beta = sqrt(*nrm2);
  for (int i = 0; i <= kMaxFgm; ++i) st->g[i] = 0.0;
  st->g[0] = st->beta;
  st->resid = st->beta;
}

// x (+)= sum_q y[q] Z[q]; xzero: x starts from 0
__global__ void __launch_bounds__(256) k_fgm_xupd(int64_t n, float* const* Z, int k, const double* __restrict__ y,
                                                  float* __restrict__ x, int xzero) {
  __shared__ float ys[kMaxFgm];
  for (int q = threadIdx.x; q < k; q += blockDim.x) ys[q] = (float)y[q];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    float xe = xzero ? 0.f : x[e];
    for (int q = 0; q < k; ++q) xe = fmaf(ys[q], Z[q][e], xe);
    x[e] = xe;
  }
}

// r = rhs - Ahat x (general 7-point matvec, FP32) and partial ||r||^2
__global__ void __launch_bounds__(kBS) k_resid_hat(Grid g, Bands<float> a, const float* __restrict__ rhs,
                                                   const float* __restrict__ x, float* __restrict__ r,
                                                   double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    const int i = (int)(col % g.nx), j = (int)(col / g.nx);
    const int64_t ie = (i == g.nx - 1) ? -(int64_t)(g.nx - 1) : 1;
    const int64_t iw = (i == 0) ? (int64_t)(g.nx - 1) : -1;
    for (int k = 0; k < g.nz; ++k) {
      const int64_t idx = (int64_t)k * g.ncol + col;
      float y = x[idx];
      y = fmaf(a.E[idx], x[idx + ie], y);
      y = fmaf(a.W[idx], x[idx + iw], y);
      if (j + 1 < g.ny) y = fmaf(a.N[idx], x[idx + g.nx], y);
      if (j > 0) y = fmaf(a.S[idx], x[idx - g.nx], y);
      if (k + 1 < g.nz) y = fmaf(a.U[idx], x[idx + g.ncol], y);
      if (k > 0) y = fmaf(a.D[idx], x[idx - g.ncol], y);
      const float rk = rhs[idx] - y;
      r[idx] = rk;
      acc += (double)(rk * rk);
    }
  }
  __shared__ double sm[kBS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) sm[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x2 = 0.0;
    for (int wi = 0; wi < kBS / 32; ++wi) x2 += sm[wi];
    part[blockIdx.x * (kMaxFgm + 1)] = x2;
  }
}

// ---------------------------------------------------------------------------
// host-side launch helpers
int fgm_grid(const Launch& L, int64_t n) {
  int64_t g = (int64_t)L.sms * 8;
  const int64_t need = (n + 255) / 256;
  if (g > need) g = need;
  if (g > kMaxGrid) g = kMaxGrid;
  return g < 1 ? 1 : (int)g;
}

// h[q] (q < nv) = <V_q, w>, into dst (device), via partials
cudaError_t fgm_multidot(const FgmWs& W, int64_t n, float* const* Vdev, int nv, const float* w, double* dst,
                         const Launch& L) {
  const int grid = fgm_grid(L, n);
  for (int q0 = 0; q0 < nv; q0 += kChunk) {
    const int nq = nv - q0 < kChunk ? nv - q0 : kChunk;
    k_mdot<<<grid, 256, 0, L.stream>>>(n, Vdev, q0, nq, w, W.part, kMaxFgm + 1);
  }
  k_psum<<<1, 64, 0, L.stream>>>(W.part, kMaxFgm + 1, grid, nv, dst);
  return cudaGetLastError();
}

// w -= sum c_q V_q; with norm: *nrm2_dst = ||w||^2
cudaError_t fgm_update(const FgmWs& W, int64_t n, float* const* Vdev, int nv, const double* c, float* w,
                       double* nrm2_dst, const Launch& L) {
  const int grid = fgm_grid(L, n);
  k_mupdate<<<grid, 256, 0, L.stream>>>(n, Vdev, nv, c, w, W.part, kMaxFgm + 1, nrm2_dst != nullptr);
  if (nrm2_dst) k_psum<<<1, 32, 0, L.stream>>>(W.part, kMaxFgm + 1, grid, 1, nrm2_dst);
  return cudaGetLastError();
}

cudaError_t fgm_scale(int64_t n, const float* x, float* y, const double* s, int inv_sqrt, const Launch& L) {
  k_scale<<<fgm_grid(L, n), 256, 0, L.stream>>>(n, x, y, s, inv_sqrt);
  return cudaGetLastError();
}

cudaError_t fgm_step(FgmState* st, int j, cudaStream_t s) {
  k_fgm_step<<<1, 32, 0, s>>>(st, j);
  return cudaGetLastError();
}

cudaError_t fgm_solve_update(FgmState* st, int64_t n, float* const* Zdev, int k, float* x, int xzero,
                             const Launch& L) {
  k_fgm_solve<<<1, 32, 0, L.stream>>>(st, k);
  k_fgm_xupd<<<fgm_grid(L, n), 256, 0, L.stream>>>(n, Zdev, k, st->y, x, xzero);
  return cudaGetLastError();
}

cudaError_t fgm_start(FgmState* st, const double* nrm2, cudaStream_t s) {
  k_fgm_start<<<1, 32, 0, s>>>(st, nrm2);
  return cudaGetLastError();
}

cudaError_t fgm_residual(const FgmWs& W, const Grid& g, const Bands<float>& a, const float* rhs, const float* x,
                         float* r, double* nrm2_dst, const Launch& L) {
  int grid = grid_for((const void*)k_resid_hat, kBS, L, L.wcol);
  k_resid_hat<<<grid, kBS, 0, L.stream>>>(g, a, rhs, x, r, W.part);
  k_psum<<<1, 32, 0, L.stream>>>(W.part, kMaxFgm + 1, grid, 1, nrm2_dst);
  return cudaGetLastError();
}

}  // namespace hz
