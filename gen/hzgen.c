/*
 * hzgen.c -- seeded synthetic Helmholtz systems on a lon-lat grid.
 *
 * This module only SYNTHESISES inputs (the operator's seven coefficient
 * bands and a right-hand side). It holds none of the solver's arithmetic:
 * no matvec, no preconditioner, no Krylov step.  Both the CPU oracle and the
 * GPU path consume its output, so the two see identical inputs.
 *
 * Operator: the 7-band, nonsymmetric, variable-coefficient structure of the
 * ENDGame pressure-correction matrix (Maynard & Walters, Sec. 2, the Helmholtz
 * system A x = b after the Schur-complement reduction): a Laplacian-like
 * 7-point stencil on (longitude, latitude, level), with horizontal weights
 * proportional to 1/(cos(phi) dlambda)^2 and 1/dphi^2 (unit sphere), vertical
 * weights proportional to 1/dz_k^2 on levels stretched quadratically from
 * 20 m to 2 km, each weight multiplied by an independent lognormal(0.1)
 * factor, a 5% skew term making A nonsymmetric, and the diagonal set to
 * -(sum of off-diagonals) + c with c = 1e-3 * max weight.
 *
 * Layout: index p = (k*ny + j)*nx + i, i (longitude) fastest.
 * Bands, in this order: C (centre), E (i+1), W (i-1), N (j+1), S (j-1),
 * U (k+1), D (k-1); coeffs[band*n + p].
 *
 * Random numbers: a counter-based generator built from the SplitMix64
 * finaliser (Steele, Lea & Flood, OOPSLA 2014), keyed by (seed, stream,
 * counter); normals by the Box-Muller transform.  Every value depends only on
 * its key, so the result is independent of the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define HZGEN_VERSION 1

static inline uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* 64 random bits for (seed, stream, counter). */
static inline uint64_t hz_bits(uint64_t seed, uint64_t stream, uint64_t ctr) {
  uint64_t k = mix64(mix64(seed) ^ ((stream + 1ull) * 0xD1B54A32D192ED03ull));
  return mix64(k ^ (ctr * 0x9E3779B97F4A7C15ull));
}

/* uniform on the open interval (0,1) with 53 random bits. */
static inline double hz_uniform(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return ((double)(hz_bits(seed, stream, ctr) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* standard normal by Box-Muller from two independent uniforms. */
static inline double hz_normal(uint64_t seed, uint64_t stream, uint64_t idx) {
  double u1 = hz_uniform(seed, stream, 2ull * idx);
  double u2 = hz_uniform(seed, stream, 2ull * idx + 1ull);
  return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

int hzgen_version(void) { return HZGEN_VERSION; }

double hzgen_uniform(uint64_t seed, uint64_t stream, uint64_t ctr) { return hz_uniform(seed, stream, ctr); }
double hzgen_normal(uint64_t seed, uint64_t stream, uint64_t idx) { return hz_normal(seed, stream, idx); }
uint64_t hzgen_bits(uint64_t seed, uint64_t stream, uint64_t ctr) { return hz_bits(seed, stream, ctr); }

/* fill out[i] = normal(seed, stream, i) for i < count (used for test vectors) */
void hzgen_normals(uint64_t seed, uint64_t stream, int64_t count, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < count; ++i) out[i] = hz_normal(seed, stream, (uint64_t)i);
}

enum { ST_E = 0, ST_W, ST_N, ST_S, ST_U, ST_D, ST_NOISE, ST_MODES };

/* layer thickness of level k, metres: 20 m at the bottom, 2 km at the top */
static double layer_dz_m(int k, int nz) {
  double s = nz > 1 ? (double)k / (double)(nz - 1) : 0.0;
  return 20.0 + 1980.0 * s * s;
}

/*
 * Operator coefficients.  z_scale converts metres to the horizontal length
 * unit (1/6.371e6 for Earth radii, 1.0 for metres).  sigma is the lognormal
 * width (0.1), skew the nonsymmetric fraction (0.05), shift_frac the
 * diagonal shift relative to the largest weight (1e-3).
 * Returns 0, or -1 on bad sizes.
 */
int hzgen_operator(int nx, int ny, int nz, uint64_t seed, double z_scale,
                   double sigma, double skew, double shift_frac, double* coeffs) {
  if (nx < 1 || ny < 1 || nz < 1 || !coeffs) return -1;
  const int64_t n = (int64_t)nx * ny * nz;
  const double dlam = 2.0 * M_PI / nx, dphi = M_PI / ny;
  double* C = coeffs;
  double* band[6];
  for (int b = 0; b < 6; ++b) band[b] = coeffs + (int64_t)(b + 1) * n;
  double wmax = 0.0;

  /* pass 1: perturbed weights w_b >= 0 stored (positive) in the band arrays */
#pragma omp parallel for schedule(static) reduction(max : wmax)
  for (int64_t p = 0; p < n; ++p) {
    const int i = (int)(p % nx);
    const int j = (int)((p / nx) % ny);
    const int k = (int)(p / ((int64_t)nx * ny));
    (void)i;
    const double phi = -0.5 * M_PI + (j + 0.5) * dphi;
    const double cl = cos(phi) * dlam;
    const double dz = layer_dz_m(k, nz) * z_scale;
    double base[6];
    base[0] = base[1] = 1.0 / (cl * cl);         /* E, W */
    base[2] = base[3] = 1.0 / (dphi * dphi);     /* N, S */
    base[4] = base[5] = 1.0 / (dz * dz);         /* U, D */
    if (j == ny - 1) base[2] = 0.0;              /* no flux across the north pole row */
    if (j == 0) base[3] = 0.0;                   /* ... nor the south */
    if (k == nz - 1) base[4] = 0.0;              /* no flux through the top */
    if (k == 0) base[5] = 0.0;                   /* ... nor the bottom */
    for (int b = 0; b < 6; ++b) {
      double w = base[b] == 0.0 ? 0.0 : base[b] * exp(sigma * hz_normal(seed, (uint64_t)b, (uint64_t)p));
      band[b][p] = w;
      if (w > wmax) wmax = w;
    }
  }
  const double c = shift_frac * wmax;
  /* pass 2: skew, sign and diagonal.  sgn = +1 for E, N, U and -1 for W, S, D */
  static const double sgn[6] = {+1.0, -1.0, +1.0, -1.0, +1.0, -1.0};
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) {
    double s = 0.0;
    for (int b = 0; b < 6; ++b) {
      double a = -band[b][p] * (1.0 - skew * sgn[b]);
      band[b][p] = a;
      s += a;
    }
    C[p] = -s + c;
  }
  return 0;
}

/*
 * Right-hand side: 16 smooth separable modes normalised to unit RMS, plus
 * noise_frac * N(0,1) white noise.  Mode q is
 *   a_q cos(m_q lam_i + th_q) cos(phi_j)^m_q cos(l_q phi_j + ps_q) cos(pi n_q (k+1/2)/nz + ch_q)
 * with a_q ~ N(0,1), m_q, l_q uniform in 0..8, n_q uniform in 0..3 and the
 * phases uniform in [0, 2 pi).  The cos^m factor keeps each mode regular at
 * the poles.
 */
#define NMODES 16
int hzgen_rhs(int nx, int ny, int nz, uint64_t seed, double noise_frac, double* b) {
  if (nx < 1 || ny < 1 || nz < 1 || !b) return -1;
  const int64_t n = (int64_t)nx * ny * nz;
  const double dlam = 2.0 * M_PI / nx, dphi = M_PI / ny;
  double amp[NMODES];
  int mq[NMODES], lq[NMODES], nq[NMODES];
  double th[NMODES], ps[NMODES], ch[NMODES];
  for (int q = 0; q < NMODES; ++q) {
    uint64_t c0 = (uint64_t)q * 16ull;
    amp[q] = sqrt(-2.0 * log(hz_uniform(seed, ST_MODES, c0))) * cos(2.0 * M_PI * hz_uniform(seed, ST_MODES, c0 + 1));
    mq[q] = (int)floor(9.0 * hz_uniform(seed, ST_MODES, c0 + 2));
    lq[q] = (int)floor(9.0 * hz_uniform(seed, ST_MODES, c0 + 3));
    nq[q] = (int)floor(4.0 * hz_uniform(seed, ST_MODES, c0 + 4));
    th[q] = 2.0 * M_PI * hz_uniform(seed, ST_MODES, c0 + 5);
    ps[q] = 2.0 * M_PI * hz_uniform(seed, ST_MODES, c0 + 6);
    ch[q] = 2.0 * M_PI * hz_uniform(seed, ST_MODES, c0 + 7);
  }
  double* X = (double*)malloc(sizeof(double) * NMODES * (size_t)nx);
  double* Y = (double*)malloc(sizeof(double) * NMODES * (size_t)ny);
  double* Z = (double*)malloc(sizeof(double) * NMODES * (size_t)nz);
  if (!X || !Y || !Z) { free(X); free(Y); free(Z); return -2; }
  for (int q = 0; q < NMODES; ++q) {
    for (int i = 0; i < nx; ++i) X[q * nx + i] = cos(mq[q] * (i * dlam) + th[q]);
    for (int j = 0; j < ny; ++j) {
      double phi = -0.5 * M_PI + (j + 0.5) * dphi;
      Y[q * ny + j] = pow(cos(phi), (double)mq[q]) * cos(lq[q] * phi + ps[q]);
    }
    for (int k = 0; k < nz; ++k) Z[q * nz + k] = amp[q] * cos(M_PI * nq[q] * (k + 0.5) / nz + ch[q]);
  }
  /* sum of squares in fixed chunks, each summed in index order, the chunk sums
     then added in chunk order: the same bits whatever the thread count (an
     OpenMP reduction would combine per-thread partials in an order that
     follows the number of threads, and so would the right-hand side) */
  const int64_t CH = (int64_t)1 << 16;
  const int64_t nch = (n + CH - 1) / CH;
  double* part = (double*)malloc(sizeof(double) * (size_t)nch);
  if (!part) { free(X); free(Y); free(Z); return -2; }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nch; ++c) {
    const int64_t p1 = (c + 1) * CH < n ? (c + 1) * CH : n;
    double sc = 0.0;
    for (int64_t p = c * CH; p < p1; ++p) {
      const int i = (int)(p % nx);
      const int j = (int)((p / nx) % ny);
      const int k = (int)(p / ((int64_t)nx * ny));
      double f = 0.0;
      for (int q = 0; q < NMODES; ++q) f += X[q * nx + i] * Y[q * ny + j] * Z[q * nz + k];
      b[p] = f;
      sc += f * f;
    }
    part[c] = sc;
  }
  double ss = 0.0;
  for (int64_t c = 0; c < nch; ++c) ss += part[c];
  free(part);
  double rms = sqrt(ss / (double)n);
  double inv = rms > 0.0 ? 1.0 / rms : 1.0;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) b[p] = b[p] * inv + noise_frac * hz_normal(seed, ST_NOISE, (uint64_t)p);
  free(X); free(Y); free(Z);
  return 0;
}
