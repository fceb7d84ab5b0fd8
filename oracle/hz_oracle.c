/*
 * hz_oracle.c -- plain, slow, serial FP64 reference for the Helmholtz solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA library: every routine
 * here is written from the paper (Maynard & Walters, "Precision of the
 * ENDGame", arXiv:1811.03852) in the simplest loop form.
 *
 * Grid and layout: nx (longitude, periodic) x ny (latitude, closed at the
 * poles) x nz (levels, closed at top and bottom); p = (k*ny + j)*nx + i.
 * Operator: 7 bands C,E,W,N,S,U,D stored band-major, A[b*n + p].
 *
 * Pins (what checks this file against something other than itself) live in
 * tests/test_oracle_*.py: dense assembled matrices with LAPACK solves,
 * banded solves, closed forms (A*1 = c*1, the one-iteration case without
 * horizontal coupling, nz = 1), manufactured solutions and brute force.
 *
 * Threads: the same source builds serial (the tests' oracle) and with OpenMP
 * (only to time the oracle on all host cores).  Only loops whose iterations
 * are independent (points, columns, vector updates) are shared out; every
 * value is computed by the same arithmetic either way.  Sums over the grid
 * (dot products, norms) run over fixed chunks of OR_CHUNK points, each summed
 * in order, and the chunk sums are added in chunk order, so the result is
 * the same bits for any number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, k) (((int64_t)(k) * ny + (j)) * nx + (i))
#define OR_CHUNK 65536

#ifdef _OPENMP
#include <omp.h>
#endif

/* threads used by the OpenMP build (1 in the serial build) */
void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

enum { B_C = 0, B_E, B_W, B_N, B_S, B_U, B_D };

int or_version(void) { return 1; }

static double dot_d(int64_t n, const double* a, const double* b);

/* ---------------------------------------------------------------------------
 * The linear system A x = b (Sec. 1, the pressure-correction equation; Sec. 2,
 * the 7-band Helmholtz matrix).  y = A x with the unscaled bands.
 * Neighbours: i+-1 wrap around (longitude is periodic); a missing j or k
 * neighbour contributes nothing (its coefficient is zero by construction).
 * ------------------------------------------------------------------------- */
void or_matvec(int nx, int ny, int nz, const double* A, const double* x, double* y) {
  const int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t p = IDX(i, j, k);
        double acc = A[B_C * n + p] * x[p];
        acc += A[B_E * n + p] * x[IDX((i + 1) % nx, j, k)];
        acc += A[B_W * n + p] * x[IDX((i + nx - 1) % nx, j, k)];
        if (j + 1 < ny) acc += A[B_N * n + p] * x[IDX(i, j + 1, k)];
        if (j > 0) acc += A[B_S * n + p] * x[IDX(i, j - 1, k)];
        if (k + 1 < nz) acc += A[B_U * n + p] * x[IDX(i, j, k + 1)];
        if (k > 0) acc += A[B_D * n + p] * x[IDX(i, j, k - 1)];
        y[p] = acc;
      }
}

/* r = b - A x and return ||r||_2 (Sec. 3, the halting residual r_i = b - A x_i). */
double or_residual(int nx, int ny, int nz, const double* A, const double* b, const double* x, double* r) {
  const int64_t n = (int64_t)nx * ny * nz;
  or_matvec(nx, ny, nz, A, x, r);
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < n; ++p) r[p] = b[p] - r[p];
  return sqrt(dot_d(n, r, r));
}

/* ---------------------------------------------------------------------------
 * Diagonal scaling outside the solver (Sec. 2, the post-conditioned system
 * D_g^-1 A C C^-1 x = D_g^-1 b):  Ahat = D^-1 A has unit diagonal, so only
 * the six off-diagonal bands are kept, Ahat[(b-1)*n + p] = A_b(p)/A_C(p).
 * ------------------------------------------------------------------------- */
void or_scale(int nx, int ny, int nz, const double* A, double* Ahat) {
  const int64_t n = (int64_t)nx * ny * nz;
  for (int b = 1; b < 7; ++b) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) Ahat[(int64_t)(b - 1) * n + p] = A[(int64_t)b * n + p] / A[p];
  }
}

/* y = Ahat x, Ahat = I + off-diagonal bands (order E,W,N,S,U,D). */
void or_matvec_hat(int nx, int ny, int nz, const double* Ah, const double* x, double* y) {
  const int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t p = IDX(i, j, k);
        double acc = x[p];
        acc += Ah[0 * n + p] * x[IDX((i + 1) % nx, j, k)];
        acc += Ah[1 * n + p] * x[IDX((i + nx - 1) % nx, j, k)];
        if (j + 1 < ny) acc += Ah[2 * n + p] * x[IDX(i, j + 1, k)];
        if (j > 0) acc += Ah[3 * n + p] * x[IDX(i, j - 1, k)];
        if (k + 1 < nz) acc += Ah[4 * n + p] * x[IDX(i, j, k + 1)];
        if (k > 0) acc += Ah[5 * n + p] * x[IDX(i, j, k - 1)];
        y[p] = acc;
      }
}

/* ---------------------------------------------------------------------------
 * Tridiagonal solve by Gaussian elimination without pivoting (the Thomas
 * algorithm) for one column of m unknowns:
 *   lo[k] x[k-1] + di[k] x[k] + up[k] x[k+1] = r[k].
 * work holds 2m doubles.  The factors are recomputed on every call.
 * ------------------------------------------------------------------------- */
void or_tridiag_solve(int m, const double* lo, const double* di, const double* up, const double* r, double* x,
                      double* work) {
  double* cprime = work;
  double* dprime = work + m;
  cprime[0] = up[0] / di[0];
  dprime[0] = r[0] / di[0];
  for (int k = 1; k < m; ++k) {
    double den = di[k] - lo[k] * cprime[k - 1];
    cprime[k] = up[k] / den;
    dprime[k] = (r[k] - lo[k] * dprime[k - 1]) / den;
  }
  x[m - 1] = dprime[m - 1];
  for (int k = m - 2; k >= 0; --k) x[k] = dprime[k] - cprime[k] * x[k + 1];
}

/* ---------------------------------------------------------------------------
 * Preconditioner C = T^-1 (Sec. 2, Ahat = L + T + U with T the vertical
 * tridiagonal part; its LU is per horizontal point, no vertical
 * decomposition).  For each column (i,j): T has sub-diagonal Ahat_D,
 * diagonal 1 and super-diagonal Ahat_U.  z = T^-1 r.
 * ------------------------------------------------------------------------- */
void or_apply_Tinv(int nx, int ny, int nz, const double* Ah, const double* r, double* z) {
  const int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel
  {
    /* one column's work arrays (per thread) */
    double* lo = (double*)malloc(sizeof(double) * 7 * (size_t)nz);
    double* di = lo + nz;
    double* up = di + nz;
    double* rc = up + nz;
    double* xc = rc + nz;
    double* wk = xc + nz;
#pragma omp for collapse(2) schedule(static)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        for (int k = 0; k < nz; ++k) {
          int64_t p = IDX(i, j, k);
          lo[k] = Ah[5 * n + p];
          di[k] = 1.0;
          up[k] = Ah[4 * n + p];
          rc[k] = r[p];
        }
        or_tridiag_solve(nz, lo, di, up, rc, xc, wk);
        for (int k = 0; k < nz; ++k) z[IDX(i, j, k)] = xc[k];
      }
    free(lo);
  }
}

/* ---------------------------------------------------------------------------
 * The paper's preconditioner (Sec. 2): a few sweeps of SOR with the vertical
 * tridiagonal T in place of the diagonal, Ahat = L + T + U,
 *   (T + omega L) x_n = (1 - omega) T x_(n-1) + omega (r - U x_(n-1)),  x_0 = 0,
 * i.e. per column x_n = (1 - omega) x_(n-1) + omega T^-1 (r - L x_n - U x_(n-1)).
 * Column order: red-black in (i, j) (colour (i + j) mod 2, red first), so the
 * horizontal neighbours of a red column are black (U) and those of a black
 * column red (L).  z = x after `sweeps` sweeps.
 * ------------------------------------------------------------------------- */
void or_apply_trisor(int nx, int ny, int nz, const double* Ah, const double* r, double* z, int sweeps,
                     double omega) {
  const int64_t n = (int64_t)nx * ny * nz;
  /* within one colour pass every column reads the values from before the pass
     (for even nx no two columns of a colour are neighbours, so this is
     Gauss-Seidel in the red-black order; for odd nx it stays well defined) */
  double* zo = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t p = 0; p < n; ++p) z[p] = 0.0;
  for (int sw = 0; sw < sweeps; ++sw)
    for (int colour = 0; colour < 2; ++colour) {
#pragma omp parallel for schedule(static)
      for (int64_t p = 0; p < n; ++p) zo[p] = z[p];
#pragma omp parallel
      {
        /* one column's work arrays (per thread) */
        double* lo = (double*)malloc(sizeof(double) * 7 * (size_t)nz);
        double* di = lo + nz;
        double* up = di + nz;
        double* rc = up + nz;
        double* xc = rc + nz;
        double* wk = xc + nz;
#pragma omp for collapse(2) schedule(static)
        for (int j = 0; j < ny; ++j)
          for (int i = 0; i < nx; ++i) {
            if (((i + j) & 1) != colour) continue;
            for (int k = 0; k < nz; ++k) {
              int64_t p = IDX(i, j, k);
              double h =
                  Ah[0 * n + p] * zo[IDX((i + 1) % nx, j, k)] + Ah[1 * n + p] * zo[IDX((i + nx - 1) % nx, j, k)];
              if (j + 1 < ny) h += Ah[2 * n + p] * zo[IDX(i, j + 1, k)];
              if (j > 0) h += Ah[3 * n + p] * zo[IDX(i, j - 1, k)];
              lo[k] = Ah[5 * n + p];
              di[k] = 1.0;
              up[k] = Ah[4 * n + p];
              rc[k] = r[p] - h;
            }
            or_tridiag_solve(nz, lo, di, up, rc, xc, wk);
            for (int k = 0; k < nz; ++k) {
              int64_t p = IDX(i, j, k);
              z[p] = (1.0 - omega) * z[p] + omega * xc[k];
            }
          }
        free(lo);
      }
    }
  free(zo);
}

/* Preconditioner used by or_bicgstab: kind 0 = T^-1, kind 1 = tri-SOR (sweeps, omega). */
static int g_pc_kind = 0, g_pc_sweeps = 3;
static double g_pc_omega = 1.5;
void or_set_precond(int kind, int sweeps, double omega) {
  g_pc_kind = kind;
  g_pc_sweeps = sweeps;
  g_pc_omega = omega;
}
static void apply_precond(int nx, int ny, int nz, const double* Ah, const double* r, double* z) {
  if (g_pc_kind == 1)
    or_apply_trisor(nx, ny, nz, Ah, r, z, g_pc_sweeps, g_pc_omega);
  else
    or_apply_Tinv(nx, ny, nz, Ah, r, z);
}

/* FP32-emulated variants: every stored value is a float, arithmetic in float. */
static void matvec_hat_f32(int nx, int ny, int nz, const float* Ah, const float* x, float* y) {
  const int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int64_t p = IDX(i, j, k);
        float acc = x[p];
        acc += Ah[0 * n + p] * x[IDX((i + 1) % nx, j, k)];
        acc += Ah[1 * n + p] * x[IDX((i + nx - 1) % nx, j, k)];
        if (j + 1 < ny) acc += Ah[2 * n + p] * x[IDX(i, j + 1, k)];
        if (j > 0) acc += Ah[3 * n + p] * x[IDX(i, j - 1, k)];
        if (k + 1 < nz) acc += Ah[4 * n + p] * x[IDX(i, j, k + 1)];
        if (k > 0) acc += Ah[5 * n + p] * x[IDX(i, j, k - 1)];
        y[p] = acc;
      }
}

static void apply_Tinv_f32(int nx, int ny, int nz, const float* Ah, const float* r, float* z) {
  const int64_t n = (int64_t)nx * ny * nz;
#pragma omp parallel
  {
    float* cp = (float*)malloc(sizeof(float) * 2 * (size_t)nz); /* per thread */
    float* dp = cp + nz;
#pragma omp for collapse(2) schedule(static)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        /* unit diagonal: den = 1 - lo*cprime */
        int64_t p0 = IDX(i, j, 0);
        cp[0] = Ah[4 * n + p0];
        dp[0] = r[p0];
        for (int k = 1; k < nz; ++k) {
          int64_t p = IDX(i, j, k);
          float lo = Ah[5 * n + p];
          float den = 1.0f - lo * cp[k - 1];
          cp[k] = Ah[4 * n + p] / den;
          dp[k] = (r[p] - lo * dp[k - 1]) / den;
        }
        z[IDX(i, j, nz - 1)] = dp[nz - 1];
        for (int k = nz - 2; k >= 0; --k) z[IDX(i, j, k)] = dp[k] - cp[k] * z[IDX(i, j, k + 1)];
      }
    free(cp);
  }
}

/* sum_p a_p b_p: each chunk of OR_CHUNK points summed in order, then the
   chunk sums in chunk order (one chunk: the plain left-to-right sum) */
static double dot_d(int64_t n, const double* a, const double* b) {
  const int64_t nc = (n + OR_CHUNK - 1) / OR_CHUNK;
  if (nc <= 1) {
    double s = 0.0;
    for (int64_t p = 0; p < n; ++p) s += a[p] * b[p];
    return s;
  }
  double* part = (double*)malloc(sizeof(double) * (size_t)nc);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t e = (c + 1) * OR_CHUNK < n ? (c + 1) * OR_CHUNK : n;
    double s = 0.0;
    for (int64_t p = c * OR_CHUNK; p < e; ++p) s += a[p] * b[p];
    part[c] = s;
  }
  double s = 0.0;
  for (int64_t c = 0; c < nc; ++c) s += part[c];
  free(part);
  return s;
}

/* dots of float vectors accumulated in double (the global sums the paper moved
   back to 64-bit, Sec. 4) */
static double dot_f(int64_t n, const float* a, const float* b) {
  const int64_t nc = (n + OR_CHUNK - 1) / OR_CHUNK;
  if (nc <= 1) {
    double s = 0.0;
    for (int64_t p = 0; p < n; ++p) s += (double)a[p] * (double)b[p];
    return s;
  }
  double* part = (double*)malloc(sizeof(double) * (size_t)nc);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t e = (c + 1) * OR_CHUNK < n ? (c + 1) * OR_CHUNK : n;
    double s = 0.0;
    for (int64_t p = c * OR_CHUNK; p < e; ++p) s += (double)a[p] * (double)b[p];
    part[c] = s;
  }
  double s = 0.0;
  for (int64_t c = 0; c < nc; ++c) s += part[c];
  free(part);
  return s;
}

/* ---------------------------------------------------------------------------
 * Right-preconditioned ("post-conditioned", Sec. 2) BiCGStab (van der Vorst
 * 1992) on Ahat y = bh with C = T^-1, halting on the recursive residual
 * ||r|| <= eta ||bh|| (Sec. 3, relative residual R).  A restart is forced
 * every `restart` iterations (Sec. 4: mandatory restart after 150) and on
 * breakdown (|rho| tiny or omega = 0).
 *
 * One iteration:
 *   rho' = <r0, r>; beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v)
 *   ph = C p; v = Ahat ph; alpha = rho'/<r0, v>; s = r - alpha v
 *   (if ||s|| <= eta ||bh||: x += alpha ph, stop)
 *   sh = C s; t = Ahat sh; omega = <t,s>/<t,t>
 *   x += alpha ph + omega sh; r = s - omega t
 * x is in/out (the initial guess on entry).  hist (may be NULL) receives the
 * recursive relative residual after each iteration (up to maxit values).
 * out[0] = iterations, out[1] = restarts, out[2] = final relative residual,
 * out[3] = status (0 converged, 1 iteration limit, 2 non-finite).
 * ------------------------------------------------------------------------- */
typedef struct {
  double iters, restarts, relres, status;
} or_info;

void or_bicgstab(int nx, int ny, int nz, const double* Ah, const double* bh, double* x, double eta, int maxit,
                 int restart, double* hist, double* out) {
  const int64_t n = (int64_t)nx * ny * nz;
  double* r = (double*)calloc((size_t)n * 8, sizeof(double));
  double *r0 = r + n, *p = r0 + n, *v = p + n, *ph = v + n, *s = ph + n, *sh = s + n, *t = sh + n;
  const double bnorm = sqrt(dot_d(n, bh, bh));
  const double stop = eta * bnorm;
  int it = 0, nrestart = 0, status = 1;
  double rnorm = 0.0;
  int fresh = 1;
  double rho = 1, alpha = 1, omega = 1;
  int since = 0;
  if (bnorm == 0.0) {
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) x[q] = 0.0;
    status = 0;
    goto done;
  }
  while (it < maxit) {
    if (fresh) { /* (re)start: r = bh - Ahat x, r0 = r, p = v = 0 */
      or_matvec_hat(nx, ny, nz, Ah, x, r);
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n; ++q) {
        r[q] = bh[q] - r[q];
        r0[q] = r[q];
        p[q] = 0.0;
        v[q] = 0.0;
      }
      rho = alpha = omega = 1.0;
      since = 0;
      fresh = 0;
      rnorm = sqrt(dot_d(n, r, r));
      if (rnorm <= stop) { status = 0; break; }
    }
    double rho1 = dot_d(n, r0, r);
    double r0n = sqrt(dot_d(n, r0, r0));
    if (fabs(rho1) <= 1e-14 * r0n * rnorm) { fresh = 1; ++nrestart; continue; }
    ++it;
    ++since;
    double beta = (rho1 / rho) * (alpha / omega);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) p[q] = r[q] + beta * (p[q] - omega * v[q]);
    apply_precond(nx, ny, nz, Ah, p, ph);
    or_matvec_hat(nx, ny, nz, Ah, ph, v);
    alpha = rho1 / dot_d(n, r0, v);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) s[q] = r[q] - alpha * v[q];
    double snorm = sqrt(dot_d(n, s, s));
    if (snorm <= stop) {
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n; ++q) x[q] += alpha * ph[q];
      rnorm = snorm;
      if (hist) hist[it - 1] = rnorm / bnorm;
      status = 0;
      break;
    }
    apply_precond(nx, ny, nz, Ah, s, sh);
    or_matvec_hat(nx, ny, nz, Ah, sh, t);
    double tt = dot_d(n, t, t);
    omega = tt > 0.0 ? dot_d(n, t, s) / tt : 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
      x[q] += alpha * ph[q] + omega * sh[q];
      r[q] = s[q] - omega * t[q];
    }
    rho = rho1;
    rnorm = sqrt(dot_d(n, r, r));
    if (hist) hist[it - 1] = rnorm / bnorm;
    if (!isfinite(rnorm)) { status = 2; break; }
    if (rnorm <= stop) { status = 0; break; }
    if (omega == 0.0 || since >= restart) { fresh = 1; ++nrestart; }
  }
done:
  if (out) {
    out[0] = it;
    out[1] = nrestart;
    out[2] = bnorm > 0 ? rnorm / bnorm : 0.0;
    out[3] = status;
  }
  free(r);
}

/* The same iteration with every vector and coefficient rounded to float and
   float arithmetic, dots accumulated in double and the scalars kept in double
   (the mixed-precision split of Sec. 3-4). Ah32 is the float copy of Ahat.
   x64 == NULL: the iterate x is a float vector too.  x64 != NULL: the paper's
   mixed-precision solver (Sec. 3: the pressure field stays 64-bit while the
   solver works in 32-bit): the iterate lives in x64 and is updated in double
   from the float vectors and the double scalars; where the iteration reads x
   (a restart's r = bh - Ahat x) it is rounded to float first.  The recursion
   itself never reads x, so without a restart both variants produce the same
   residuals. */
static void bicgstab_f32(int nx, int ny, int nz, const float* Ah, const float* bh, float* x, double* x64, double eta,
                         int maxit, int restart, double* hist, double* out) {
  const int64_t n = (int64_t)nx * ny * nz;
  float* r = (float*)calloc((size_t)n * 9, sizeof(float));
  float *r0 = r + n, *p = r0 + n, *v = p + n, *ph = v + n, *s = ph + n, *sh = s + n, *t = sh + n, *xf = t + n;
  const double bnorm = sqrt(dot_f(n, bh, bh));
  const double stop = eta * bnorm;
  int it = 0, nrestart = 0, status = 1;
  double rnorm = 0.0;
  int fresh = 1;
  double rho = 1, alpha = 1, omega = 1;
  int since = 0;
  if (bnorm == 0.0) {
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
      if (x64)
        x64[q] = 0.0;
      else
        x[q] = 0.0f;
    }
    status = 0;
    goto done;
  }
  while (it < maxit) {
    if (fresh) {
      const float* xr = x;
      if (x64) {
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; ++q) xf[q] = (float)x64[q];
        xr = xf;
      }
      matvec_hat_f32(nx, ny, nz, Ah, xr, r);
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n; ++q) {
        r[q] = bh[q] - r[q];
        r0[q] = r[q];
        p[q] = 0.0f;
        v[q] = 0.0f;
      }
      rho = alpha = omega = 1.0;
      since = 0;
      fresh = 0;
      rnorm = sqrt(dot_f(n, r, r));
      if (rnorm <= stop) { status = 0; break; }
    }
    double rho1 = dot_f(n, r0, r);
    double r0n = sqrt(dot_f(n, r0, r0));
    if (fabs(rho1) <= 1e-14 * r0n * rnorm) { fresh = 1; ++nrestart; continue; }
    ++it;
    ++since;
    float beta = (float)((rho1 / rho) * (alpha / omega));
    float om = (float)omega;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) p[q] = r[q] + beta * (p[q] - om * v[q]);
    apply_Tinv_f32(nx, ny, nz, Ah, p, ph);
    matvec_hat_f32(nx, ny, nz, Ah, ph, v);
    alpha = rho1 / dot_f(n, r0, v);
    float al = (float)alpha;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) s[q] = r[q] - al * v[q];
    double snorm = sqrt(dot_f(n, s, s));
    if (snorm <= stop) {
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n; ++q) {
        if (x64)
          x64[q] += alpha * (double)ph[q];
        else
          x[q] += al * ph[q];
      }
      rnorm = snorm;
      if (hist) hist[it - 1] = rnorm / bnorm;
      status = 0;
      break;
    }
    apply_Tinv_f32(nx, ny, nz, Ah, s, sh);
    matvec_hat_f32(nx, ny, nz, Ah, sh, t);
    double tt = dot_f(n, t, t);
    omega = tt > 0.0 ? dot_f(n, t, s) / tt : 0.0;
    om = (float)omega;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
      if (x64)
        x64[q] += alpha * (double)ph[q] + omega * (double)sh[q];
      else
        x[q] += al * ph[q] + om * sh[q];
      r[q] = s[q] - om * t[q];
    }
    rho = rho1;
    rnorm = sqrt(dot_f(n, r, r));
    if (hist) hist[it - 1] = rnorm / bnorm;
    if (!isfinite(rnorm)) { status = 2; break; }
    if (rnorm <= stop) { status = 0; break; }
    if (omega == 0.0 || since >= restart) { fresh = 1; ++nrestart; }
  }
done:
  if (out) {
    out[0] = it;
    out[1] = nrestart;
    out[2] = bnorm > 0 ? rnorm / bnorm : 0.0;
    out[3] = status;
  }
  free(r);
}

void or_bicgstab_f32(int nx, int ny, int nz, const float* Ah, const float* bh, float* x, double eta, int maxit,
                     int restart, double* hist, double* out) {
  bicgstab_f32(nx, ny, nz, Ah, bh, x, NULL, eta, maxit, restart, hist, out);
}

/* the paper's mixed-precision solver: x in double, everything else float */
void or_bicgstab_mp(int nx, int ny, int nz, const float* Ah, const float* bh, double* x, double eta, int maxit,
                    int restart, double* hist, double* out) {
  bicgstab_f32(nx, ny, nz, Ah, bh, NULL, x, eta, maxit, restart, hist, out);
}

/* ---------------------------------------------------------------------------
 * Outer loop judged by the true FP64 residual R = ||b - A x|| / ||b|| (Sec. 3,
 * the relative residual and halting criterion R < R_c), with the inner
 * correction solve on the scaled system Ahat d = D^-1 r:
 *   mode 0: inner solve in FP64;
 *   mode 1: inner solve in FP32 (mixed precision; iterative refinement wins
 *           back the digits below the 32-bit limit eps_32 of Sec. 3);
 *   mode 2: the paper's mixed-precision solver (Sec. 3): one solve with x in
 *           FP64 and everything else in FP32, to eta, and no refinement (the
 *           outer loop stops after it and reports R).
 * x is in/out (initial guess).  outer_hist (may be NULL, max_outer+1 values)
 * receives R before each outer step and after the last.  Ah32_in (may be
 * NULL): the FP32 operator of the inner solves of modes 1 and 2 ([6][n],
 * E,W,N,S,U,D), instead of the float rounding of Ahat.
 * out[0] = outer iterations, out[1] = total inner iterations,
 * out[2] = final true R, out[3] = status (0 ok, 1 not converged, 2 non-finite),
 * out[4] = total restarts.
 * ------------------------------------------------------------------------- */
void or_solve(int nx, int ny, int nz, const double* A, const double* b, double* x, int mode, double tol,
              double eta, int max_outer, int max_inner, int restart, double* outer_hist, double* out,
              const float* Ah32_in) {
  const int64_t n = (int64_t)nx * ny * nz;
  double* Ah = (double*)malloc(sizeof(double) * 6 * (size_t)n);
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  float* Ah32 = NULL;
  float *r32 = NULL, *d32 = NULL;
  or_scale(nx, ny, nz, A, Ah);
  if (mode == 1 || mode == 2) {
    Ah32 = (float*)malloc(sizeof(float) * 6 * (size_t)n);
    r32 = (float*)malloc(sizeof(float) * (size_t)n);
    d32 = (float*)malloc(sizeof(float) * (size_t)n);
    /* the FP32 inner operator: the float rounding of Ahat, or the caller's
       (e.g. with the horizontal bands stored in 16 bits) */
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < 6 * n; ++q) Ah32[q] = Ah32_in ? Ah32_in[q] : (float)Ah[q];
  }
  const double bnorm = sqrt(dot_d(n, b, b));
  int outer = 0, inner_total = 0, status = 1, restarts = 0;
  double R = 0.0;
  for (;;) {
    double rn = or_residual(nx, ny, nz, A, b, x, r);
    R = bnorm > 0 ? rn / bnorm : rn;
    if (outer_hist) outer_hist[outer] = R;
    if (!isfinite(R)) { status = 2; break; }
    if (R <= tol) { status = 0; break; }
    if (outer >= max_outer) { status = 1; break; }
    double info[4];
    if (mode == 2) {
      /* the paper's mixed-precision solver: one solve, x kept in double */
      for (int64_t q = 0; q < n; ++q) {
        r32[q] = (float)(r[q] / A[q]);
        d[q] = 0.0;
      }
      or_bicgstab_mp(nx, ny, nz, Ah32, r32, d, eta, max_inner, restart, NULL, info);
      for (int64_t q = 0; q < n; ++q) x[q] += d[q];
      max_outer = outer + 1; /* no refinement */
    } else if (mode == 1) {
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n; ++q) {
        r32[q] = (float)(r[q] / A[q]);
        d32[q] = 0.0f;
      }
      or_bicgstab_f32(nx, ny, nz, Ah32, r32, d32, eta, max_inner, restart, NULL, info);
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n; ++q) x[q] += (double)d32[q];
    } else {
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n; ++q) {
        r[q] = r[q] / A[q];
        d[q] = 0.0;
      }
      or_bicgstab(nx, ny, nz, Ah, r, d, eta, max_inner, restart, NULL, info);
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n; ++q) x[q] += d[q];
    }
    inner_total += (int)info[0];
    restarts += (int)info[1];
    ++outer;
  }
  if (out) {
    out[0] = outer;
    out[1] = inner_total;
    out[2] = R;
    out[3] = status;
    out[4] = restarts;
  }
  free(Ah); free(r); free(d); free(Ah32); free(r32); free(d32);
}

/* deterministic-order FP64 dot (for reference sums in tests) */
double or_dot(int64_t n, const double* a, const double* b) { return dot_d(n, a, b); }
