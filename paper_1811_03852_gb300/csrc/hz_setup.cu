// hz_setup.cu -- operator setup and the outer FP64 true residual on sm_103a.
//
// Setup (once per operator, i.e. once per model time step, since the matrix
// changes every step -- Maynard & Walters Sec. 2): the diagonal scaling
// Ahat = D^-1 A applied outside the solver (Sec. 2, post-conditioned system)
// in FP64 and FP32, and the LU factors of the per-column tridiagonal part T
// of Ahat (Sec. 2: pre-computed at each horizontal point, no vertical
// decomposition).  With unit diagonal, the Thomas factors are
//   den_k = 1 - a_k c'_(k-1),  m_k = 1/den_k,  l_k = a_k m_k,  c'_k = u_k m_k
// (a = D band, u = U band of Ahat).  The FP32 factors are those of the
// FP32-rounded T, computed in FP64 and rounded once.
//
// True residual (Sec. 3, r_i = b - A x_i and R = ||r_i||/||b||): FP64 with the
// unscaled bands, fused with the refinement update x <- x + d and with the
// scaling/cast of the next inner right-hand side D^-1 r.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "hz_internal.cuh"

namespace hz {

__global__ void __launch_bounds__(kBS) k_setup(Grid g, const double* __restrict__ A7, SetupOut o) {
  const int64_t n = g.n;
  int err = 0;
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < g.ncol; col += (int64_t)gridDim.x * kBS) {
    const int j = (int)(col / g.nx);
    double cp64 = 0.0, cp32 = 0.0;
    for (int k = 0; k < g.nz; ++k) {
      const int64_t idx = (int64_t)k * g.ncol + col;
      const double C = A7[idx];
      if (!(C != 0.0) || !isfinite(C)) err |= 1;
      const double inv = 1.0 / C;
      double ah[6];
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        const double ab = A7[(int64_t)(b + 1) * n + idx];
        if (!isfinite(ab)) err |= 1;
        ah[b] = ab * inv;
      }
      if (j == g.ny - 1 && A7[3 * n + idx] != 0.0) err |= 2;  // N across the pole
      if (j == 0 && A7[4 * n + idx] != 0.0) err |= 2;           // S across the pole
      if (k == g.nz - 1 && A7[5 * n + idx] != 0.0) err |= 2;    // U through the top
      if (k == 0 && A7[6 * n + idx] != 0.0) err |= 2;           // D through the bottom
#pragma unroll
      for (int b = 0; b < 6; ++b) {
        o.ah64[(int64_t)b * n + idx] = ah[b];
        o.ah32[(int64_t)b * n + idx] = (float)ah[b];
      }
      o.invc[idx] = inv;
      // LU of the unit-diagonal tridiagonal T (FP64)
      const double lo = ah[5], up = ah[4];
      const double den = 1.0 - lo * cp64;
      if (!(den != 0.0) || !isfinite(den)) err |= 4;
      const double m = 1.0 / den;
      cp64 = up * m;
      o.th64[idx] = m;
      o.th64[n + idx] = lo * m;
      o.th64[2 * n + idx] = cp64;
      // LU of the FP32-rounded T, rounded once
      const double lo32 = (double)(float)lo, up32 = (double)(float)up;
      const double den32 = 1.0 - lo32 * cp32;
      if (!(den32 != 0.0) || !isfinite(den32)) err |= 4;
      const double m32 = 1.0 / den32;
      cp32 = up32 * m32;
      o.th32[idx] = (float)m32;
      o.th32[n + idx] = (float)(lo32 * m32);
      o.th32[2 * n + idx] = (float)cp32;
    }
  }
  if (err) atomicOr(o.err, err);
}

cudaError_t launch_setup(const Grid& g, const double* A7, SetupOut o, const Launch& L) {
  k_setup<<<grid_for((const void*)k_setup, kBS, L, L.wcol), kBS, 0, L.stream>>>(g, A7, o);
  return cudaGetLastError();
}

// 16-bit copies of the horizontal bands E, W, N, S of Ahat (rows 0..3 of ah64),
// rounded to nearest even: BF16 from the FP32 rounding of the FP64 value (the
// FP32 operator's value, rounded once more), FP16 directly from the FP64 value
__global__ void __launch_bounds__(256) k_h16(int64_t n, const double* __restrict__ ah64, uint16_t* __restrict__ out,
                                             int64_t stride, int fmt) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 4 * n; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / n, p = q - b * n;
    const double v = ah64[q];
    uint16_t h;
    if (fmt == HB_BF16)
      h = __bfloat16_as_ushort(__float2bfloat16_rn((float)v));
    else
      h = __half_as_ushort(__double2half(v));
    out[b * stride + p] = h;
  }
}

cudaError_t launch_h16(const Grid& g, const double* ah64, uint16_t* out, int64_t stride, int fmt, const Launch& L) {
  k_h16<<<grid_for((const void*)k_h16, 256, L, (4 * g.n + 255) / 256), 256, 0, L.stream>>>(g.n, ah64, out, stride,
                                                                                          fmt);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// r = b - A x in FP64 with x = xin + delta (either may be absent = 0).
// Writes xout = x (if given; never the buffer it reads), rhs = D^-1 r in D's
// precision, r_out (optional), and reduces ||r||^2, ||b||^2, ||rhs||^2.  The
// last block stores them in the control block and resets it for the next
// inner solve (tolerance eta relative to ||rhs||).  The correction delta is in
// DD: the inner precision D, or FP64 when the inner iterate was kept in FP64
// (the paper's mixed-precision solver).
template <typename D, typename DD, bool HAS_X, bool HAS_D>
__global__ void __launch_bounds__(kBS) k_residual(Grid g, const double* __restrict__ A7,
                                                  const double* __restrict__ invc, const double* __restrict__ b,
                                                  const double* __restrict__ xin, double* __restrict__ xout,
                                                  const DD* __restrict__ delta, D* __restrict__ rhs,
                                                  double* __restrict__ r_out, Ctl* ctl, Red red) {
  const int64_t n = g.n, ncol = g.ncol;
  // the inner correction is used only if the inner solve wrote it and it is finite
  const bool use_d = HAS_D && ctl->state != ST_NONFINITE && ctl->xzero == 0;
  auto X = [&](int64_t q) -> double {
    double v = 0.0;
    if (HAS_X) v = xin[q];
    if (HAS_D && use_d) v += (double)delta[q];
    return v;
  };
  const double* __restrict__ Cb = A7;
  const double* __restrict__ Eb = A7 + n;
  const double* __restrict__ Wb = A7 + 2 * n;
  const double* __restrict__ Nb = A7 + 3 * n;
  const double* __restrict__ Sb = A7 + 4 * n;
  const double* __restrict__ Ub = A7 + 5 * n;
  const double* __restrict__ Db = A7 + 6 * n;
  double rr = 0.0, bb = 0.0, hh = 0.0;
  for (int64_t col = (int64_t)blockIdx.x * kBS + threadIdx.x; col < ncol; col += (int64_t)gridDim.x * kBS) {
    const int i = (int)(col % g.nx);
    const int j = (int)(col / g.nx);
    const int64_t ie = (i == g.nx - 1) ? -(int64_t)(g.nx - 1) : 1;
    const int64_t iw = (i == 0) ? (int64_t)(g.nx - 1) : -1;
    const bool hn = j + 1 < g.ny, hs = j > 0;
    double xm = 0.0, xc = 0.0, xp = 0.0;
    if (HAS_X || HAS_D) {
      xc = X(col);
      xp = g.nz > 1 ? X(ncol + col) : 0.0;
    }
    double crr = 0.0, cbb = 0.0, chh = 0.0;
    for (int k = 0; k < g.nz; ++k) {
      const int64_t idx = (int64_t)k * ncol + col;
      double ax = 0.0;
      if (HAS_X || HAS_D) {
        ax = Cb[idx] * xc;
        ax = fma(Eb[idx], X(idx + ie), ax);
        ax = fma(Wb[idx], X(idx + iw), ax);
        if (hn) ax = fma(Nb[idx], X(idx + g.nx), ax);
        if (hs) ax = fma(Sb[idx], X(idx - g.nx), ax);
        if (k + 1 < g.nz) ax = fma(Ub[idx], xp, ax);
        if (k > 0) ax = fma(Db[idx], xm, ax);
        if (xout) xout[idx] = xc;
      }
      const double bv = b[idx];
      const double r = bv - ax;
      if (r_out) r_out[idx] = r;
      D h;
      if (sizeof(D) == 4) {
        h = (D)__fmul_rn((float)r, __frcp_rn((float)Cb[idx]));
      } else {
        h = (D)(r * invc[idx]);
      }
      rhs[idx] = h;
      crr = fma(r, r, crr);
      cbb = fma(bv, bv, cbb);
      chh = fma((double)h, (double)h, chh);
      if (HAS_X || HAS_D) {
        xm = xc;
        xc = xp;
        xp = (k + 2 < g.nz) ? X(idx + 2 * ncol) : 0.0;
      }
    }
    rr += crr;
    bb += cbb;
    hh += chh;
  }
  double vv[3] = {rr, bb, hh}, out[3];
  if (grid_reduce<3>(vv, red, out)) {
    ctl->res_rr = out[0];
    ctl->res_bb = out[1];
    ctl->res_hh = out[2];
    ctl->last_rnorm2 = ctl->rnorm2;
    ctl->last_bnorm2 = ctl->bnorm2;
    ctl->last_iter = HAS_D ? ctl->iter : 0;
    ctl->last_restarts = HAS_D ? ctl->restarts : 0;
    ctl->last_state = ctl->state;
    if (HAS_D) ctl->hist_off += ctl->iter;
    const double h2 = out[2];
    ctl->bnorm2 = h2;
    ctl->stop2 = ctl->eta * ctl->eta * h2;
    ctl->rho = h2;
    ctl->r0norm2 = h2;
    ctl->rnorm2 = h2;
    ctl->snorm2 = 0.0;
    ctl->alpha = 1.0;
    ctl->omega = 1.0;
    ctl->beta = 0.0;
    ctl->iter = 0;
    ctl->since = 0;
    ctl->restarts = 0;
    ctl->fresh = 1;
    ctl->rsel = 0;
    ctl->r0sel = 0;
    ctl->xzero = 1;
    ctl->bodies = 0;
    ctl->state = !isfinite(h2) ? ST_NONFINITE : (h2 > 0.0 ? ST_RUNNING : ST_CONVERGED);
  }
}

template <typename D, typename DD>
cudaError_t launch_residual_t(const Grid& g, const double* A7, const double* invc, const double* b,
                              const double* xin, double* xout, const DD* delta, D* rhs, double* r_out, Ctl* ctl,
                              Red red, const Launch& L) {
  const bool hx = xin != nullptr, hd = delta != nullptr;
  if (hx && hd)
    k_residual<D, DD, true, true><<<grid_for((const void*)k_residual<D, DD, true, true>, kBS, L, L.wcol), kBS, 0,
                                    L.stream>>>(g, A7, invc, b, xin, xout, delta, rhs, r_out, ctl, red);
  else if (hx)
    k_residual<D, DD, true, false><<<grid_for((const void*)k_residual<D, DD, true, false>, kBS, L, L.wcol), kBS, 0,
                                     L.stream>>>(g, A7, invc, b, xin, xout, delta, rhs, r_out, ctl, red);
  else if (hd)
    k_residual<D, DD, false, true><<<grid_for((const void*)k_residual<D, DD, false, true>, kBS, L, L.wcol), kBS, 0,
                                     L.stream>>>(g, A7, invc, b, xin, xout, delta, rhs, r_out, ctl, red);
  else
    k_residual<D, DD, false, false><<<grid_for((const void*)k_residual<D, DD, false, false>, kBS, L, L.wcol), kBS,
                                      0, L.stream>>>(g, A7, invc, b, xin, xout, delta, rhs, r_out, ctl, red);
  return cudaGetLastError();
}

template <typename D>
cudaError_t launch_residual(const Grid& g, const double* A7, const double* invc, const double* b, const double* xin,
                            double* xout, const D* delta, D* rhs, double* r_out, int mode, Ctl* ctl, Red red,
                            const Launch& L) {
  (void)mode;
  return launch_residual_t<D, D>(g, A7, invc, b, xin, xout, delta, rhs, r_out, ctl, red, L);
}

cudaError_t launch_residual_x64(const Grid& g, const double* A7, const double* invc, const double* b,
                                const double* xin, double* xout, const double* delta, float* rhs, Ctl* ctl, Red red,
                                const Launch& L) {
  return launch_residual_t<float, double>(g, A7, invc, b, xin, xout, delta, rhs, nullptr, ctl, red, L);
}

void warm_launch_kernels(const Launch& L) {
  grid_for((const void*)k_setup, kBS, L, 1);
  grid_for((const void*)k_h16, 256, L, 1);
#define HZ_WARM_RES(D, DD)                                               \
  grid_for((const void*)k_residual<D, DD, true, true>, kBS, L, 1);       \
  grid_for((const void*)k_residual<D, DD, true, false>, kBS, L, 1);      \
  grid_for((const void*)k_residual<D, DD, false, true>, kBS, L, 1);      \
  grid_for((const void*)k_residual<D, DD, false, false>, kBS, L, 1);
  HZ_WARM_RES(float, float)
  HZ_WARM_RES(double, double)
  HZ_WARM_RES(float, double)
#undef HZ_WARM_RES
}

template cudaError_t launch_residual<float>(const Grid&, const double*, const double*, const double*, const double*,
                                            double*, const float*, float*, double*, int, Ctl*, Red, const Launch&);
template cudaError_t launch_residual<double>(const Grid&, const double*, const double*, const double*, const double*,
                                             double*, const double*, double*, double*, int, Ctl*, Red,
                                             const Launch&);

}  // namespace hz
