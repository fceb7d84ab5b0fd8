/*
 * hz.h -- C ABI of the GB300 (sm_103a) mixed-precision Helmholtz solver.
 *
 * The solver computes x with ||b - A x||_2 / ||b||_2 <= tol for the ENDGame
 * pressure-correction system A x = b (Maynard & Walters, "Precision of the
 * ENDGame", arXiv:1811.03852: Sec. 1 eq. LinearSys; Sec. 2 eq. Helmholtz,
 * a 7-band, nonsymmetric, variable-coefficient matrix on a lon-lat grid with
 * vertical levels).  The method is the paper's post-conditioned BiCGStab on
 * the diagonally scaled system D^-1 A (Sec. 2) with the per-column vertical
 * tridiagonal part T of D^-1 A as preconditioner (Sec. 2, pre-computed LU of
 * T at each horizontal point), a mandatory restart every 150 iterations
 * (Sec. 4), FP64 global sums (Sec. 4), and -- to reach residuals below the
 * 32-bit limit of Sec. 3 -- an outer FP64 iterative-refinement loop around an
 * FP32 inner solve.
 *
 * Conventions for every entry point
 *  - Grid: nx (longitude, periodic) x ny (latitude; rows 0 and ny-1 are the
 *    polar rows, no flux across them) x nz (levels; no flux through the top
 *    and bottom).  Arrays are C-ordered [nz][ny][nx], i (longitude) fastest;
 *    point p = (k*ny + j)*nx + i.
 *  - Operator coefficients: 7 bands, band-major [7][nz][ny][nx], order
 *    C (centre), E (i+1), W (i-1), N (j+1), S (j-1), U (k+1), D (k-1).  Row p
 *    of A x is C x_p + E x_(i+1) + W x_(i-1) + N x_(j+1) + S x_(j-1) +
 *    U x_(k+1) + D x_(k-1).  N must be 0 on j = ny-1, S on j = 0, U on
 *    k = nz-1 and D on k = 0; C must be finite and nonzero.
 *  - "host or device" pointers: the library asks the CUDA runtime which kind
 *    a pointer is; host buffers are copied on the operator's stream.
 *  - Ownership: the caller owns every array it passes; the library keeps its
 *    own copies of what it needs after the call returns.  Handles are owned
 *    by the library until destroyed.
 *  - All GPU work is ordered on the stream given at create time.  No
 *    exception crosses the ABI; every call returns an hz_status.
 *  - Thread safety: one operator per host thread at a time.
 */
#ifndef HZ_H_
#define HZ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HZ_ABI_VERSION 4

typedef struct hz_op_s* hz_op;

typedef enum {
  HZ_OK = 0,
  HZ_ERR_INVALID = 1,        /* bad argument or operator (sizes, boundary coefficients, zero diagonal) */
  HZ_ERR_CUDA = 2,           /* a CUDA runtime call failed; hz_last_error() has the text */
  HZ_ERR_OOM = 3,            /* device allocation failed */
  HZ_ERR_NOT_CONVERGED = 4,  /* iteration limits reached; x holds the best iterate */
  HZ_ERR_BREAKDOWN = 5,      /* Krylov breakdown could not be cured by restarting */
  HZ_ERR_NONFINITE = 6,      /* a non-finite value appeared; x holds the last finite iterate */
  HZ_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up */
  HZ_ERR_UNSUPPORTED = 8     /* valid request this build does not provide */
} hz_status;

/* Outer/inner precision split (Sec. 3: R_c >> eps_32 allows 32-bit work). */
typedef enum {
  HZ_MODE_FP64 = 0,     /* inner BiCGStab in FP64: the double-precision baseline */
  HZ_MODE_MIXED_IR = 1, /* inner BiCGStab in FP32, outer FP64 residual and update */
  HZ_MODE_PAPER_MP = 2, /* the paper's mixed-precision solver (Sec. 3): one BiCGStab solve with the iterate
                           x in FP64 and every other vector, coefficient and preconditioner value in FP32,
                           halting when its recursive residual of the scaled system falls below tol
                           (inner_tol if given); no refinement.  The status is that halting test's (HZ_OK, or
                           HZ_ERR_NOT_CONVERGED after max_inner iterations, or HZ_ERR_NONFINITE); the report's
                           true_rel_residual is the FP64 R = ||b - A x|| / ||b|| of the x returned, which
                           may differ from the scaled recursive residual.  BiCGStab with HZ_PRE_TRI or
                           HZ_PRE_TRISOR. */
  HZ_MODE_PAPER_DP = 3  /* its 64-bit counterpart in the paper's comparison (Sec. 4, Table 1): the same single
                           solve, halting test and report, everything in FP64 */
} hz_mode;

typedef enum { HZ_PREC_FP64 = 0, HZ_PREC_FP32 = 1 } hz_prec;

typedef enum {
  HZ_PRE_TRI = 0,    /* C = T^-1, the per-column tridiagonal solve */
  HZ_PRE_TRI_NN = 1, /* T^-1 followed by the learned conv-net correction (flexible Krylov only) */
  HZ_PRE_TRISOR = 2  /* tri-SOR (Sec. 2): sor_sweeps red-black sweeps of
                        x_n = (1-w) x_(n-1) + w T^-1 (r - L x_n - U x_(n-1)), w = sor_omega,
                        from x_0 = 0; red = columns with (i + j) even, first.
                        BiCGStab only; needs nx even (HZ_ERR_UNSUPPORTED otherwise). */
} hz_precond;

typedef enum { HZ_KRYLOV_BICGSTAB = 0, HZ_KRYLOV_FGMRES = 1 } hz_krylov;

/* Solve parameters (host struct).  Fill with hz_default_params first. */
typedef struct {
  double tol;        /* target true relative residual ||b - A x|| / ||b||   (default 1e-8) */
  double inner_tol;  /* inner relative tolerance eta on the scaled system (0: default, 1e-4 mixed; tol in FP64 mode) */
  int mode;          /* hz_mode (default HZ_MODE_MIXED_IR) */
  int precond;       /* hz_precond (default HZ_PRE_TRI) */
  int krylov;        /* hz_krylov (default HZ_KRYLOV_BICGSTAB) */
  int max_outer;     /* refinement steps (default 10) */
  int max_inner;     /* inner iterations per refinement step (default 1000) */
  int restart;       /* forced BiCGStab restart period (default 150, Sec. 4) */
  int fgmres_m;      /* FGMRES restart length (default 30) */
  int use_graph;     /* 1: inner loop runs on the device inside a CUDA graph (default); 0: host-driven */
  int record_history;/* 1: keep the inner recursive residual after every iteration (hz_get_history) */
  int sor_sweeps;    /* HZ_PRE_TRISOR: sweeps per application, 1..64 (default 3, Sec. 2) */
  double sor_omega;  /* HZ_PRE_TRISOR: relaxation factor, 0 < w < 2 (default 1.5, Sec. 2) */
  int dot_fp32;      /* FP32 inner solves only: 1 sums every inner dot product in FP32 (per thread, block and
                        grid), the 32-bit global sums the paper started from (Sec. 4); 0 (default): FP32 partial
                        sums within a column batch, FP64 across them (the paper's 64-bit global sums).  With
                        HZ_MODE_FP64 or HZ_MODE_PAPER_DP: HZ_ERR_UNSUPPORTED.  FGMRES ignores it. */
  int nn_window;     /* HZ_PRE_TRI_NN: the learned stage is dropped for plain T^-1 (info->fallbacks) when the
                        FGMRES residual estimate exceeds its start or is above nn_factor times its value
                        nn_window steps earlier (default 10; 0: one restart cycle, fgmres_m steps) */
  double nn_factor;  /* in (0, 1] (default 0.5: the estimate must halve within the window) */
} hz_solve_params;

/* Solve report (host struct). */
typedef struct {
  int status;                 /* hz_status of the solve */
  int outer_iters;            /* refinement steps taken */
  int inner_iters;            /* total inner Krylov iterations */
  int restarts;               /* inner restarts (periodic + breakdown) */
  int fallbacks;              /* learned-stage fallbacks to plain T^-1 */
  int fp64_retries;           /* mixed BiCGStab only: 1 if a refinement step stalled (R not halved) or its
                                 FP32 inner solve overflowed, after which the remaining inner solves ran in
                                 FP64 from the current x; a later stall returns HZ_ERR_NOT_CONVERGED */
  double true_rel_residual;   /* final ||b - A x|| / ||b|| in FP64 (Sec. 3, eq. residual) */
  double scaled_rel_residual; /* last inner recursive residual relative to its right-hand side */
  double seconds;             /* device time of the solve */
  long long kernel_launches;  /* CUDA kernels launched by the solve */
} hz_solve_info;

int hz_version(void);
const char* hz_status_str(int status);
/* Text of the last CUDA failure seen by this thread ("" if none). */
const char* hz_last_error(void);
void hz_default_params(hz_solve_params* params);

/*
 * Create an operator from the seven coefficient bands (Sec. 2, eq. Helmholtz).
 * coeffs: host or device, 7*nx*ny*nz doubles, layout above; read during the
 * call only.  stream: a cudaStream_t (NULL = legacy default stream).
 * Work done: copy of A in FP64 (for the true residual), the diagonal scaling
 * D^-1 A in FP32 and FP64 (Sec. 2: applied outside the solver), and the
 * per-column LU factors of T in FP32 and FP64 (Sec. 2).
 * Errors: HZ_ERR_INVALID for nx<1, ny<1, nz<1, nz>HZ_MAX_LEVELS, a zero or
 * non-finite diagonal, a nonzero coefficient pointing across a pole or the
 * top/bottom, or a tridiagonal factor that breaks down; HZ_ERR_OOM.
 * On error *out is NULL.
 */
#define HZ_MAX_LEVELS 4096
int hz_op_create(int nx, int ny, int nz, const double* coeffs, void* stream, hz_op* out);

/* Replace the coefficients (a new time step: the matrix changes every step,
   Sec. 2) and redo the scaling and factorisation.  Same rules as create. */
int hz_op_update(hz_op op, const double* coeffs);

/* Release an operator and all its device memory.  NULL is accepted. */
int hz_op_destroy(hz_op op);

/* Grid of an operator. */
int hz_op_dims(hz_op op, int* nx, int* ny, int* nz);

/*
 * Solve A x = b to params->tol in the true FP64 relative residual.
 * b: host or device, n doubles.  x0: host or device initial guess, or NULL
 * for zero.  x: host or device output, n doubles; may alias x0.
 * params: NULL for defaults.  info: host, may be NULL; when given, the call
 * waits for the solve to finish and fills it (it always does so anyway,
 * since the outer loop reads the residual on the host).
 * Returns HZ_OK, HZ_ERR_NOT_CONVERGED (x = best iterate), HZ_ERR_NONFINITE
 * (x = last finite iterate), HZ_ERR_INVALID, HZ_ERR_CUDA.
 * Stagnation: a refinement step that does not halve R counts as a stall; two
 * in a row return HZ_ERR_NOT_CONVERGED.  In mixed mode with BiCGStab the first
 * stall (or an FP32 inner solve that overflows while the FP64 residual stays
 * finite) is retried once with FP64 inner solves for the rest of the solve
 * (info->fp64_retries), so a right-hand side outside the 32-bit range still
 * converges.
 */
int hz_solve(hz_op op, const double* b, const double* x0, double* x, const hz_solve_params* params,
             hz_solve_info* info);

/*
 * Solve nsys systems: independent systems (each with its own operator and
 * grid) and/or several right-hand sides of one operator (an operator may
 * appear more than once; each further occurrence gets its own work vectors,
 * allocated on first use and kept by the operator).  b[s], x0[s] (may be
 * NULL) and x[s] follow hz_solve's rules (device pointers only).
 * 1 <= nsys <= 64, operators sharing one stream; mixed mode with BiCGStab and
 * T^-1 only (else HZ_ERR_UNSUPPORTED).  infos: host array of nsys reports,
 * may be NULL.  Returns the worst status.
 *
 * Strategies (hz_solve_batched_ex; hz_solve_batched = HZ_BATCH_AUTO):
 *   HZ_BATCH_PERSISTENT: the whole solve of every system -- FP64 residuals,
 *     FP32 inner BiCGStab, refinement updates and the per-system tests on
 *     tol, max_outer and stagnation -- in ONE persistent cooperative launch,
 *     phases separated by a grid barrier whose waits are bounded
 *     (HZ_ERR_TIMEOUT instead of a hang); systems that are done are masked
 *     out.  With params->use_graph the launch is captured in a CUDA graph and
 *     replayed when the same systems (operators, b, x0, x) come again.
 *   HZ_BATCH_SEQUENTIAL: hz_solve on each system in turn (graph-captured
 *     inner loops, each kernel at its own occupancy); same arithmetic per
 *     system as a single solve.
 *   HZ_BATCH_AUTO: SEQUENTIAL when every system has at least 2^20 points (one
 *     system then fills the GPU), else PERSISTENT.
 * Any other strategy value: HZ_ERR_INVALID.
 */
#define HZ_BATCH_AUTO 0
#define HZ_BATCH_PERSISTENT 1
#define HZ_BATCH_SEQUENTIAL 2
int hz_solve_batched(int nsys, const hz_op* ops, const double* const* b, const double* const* x0, double* const* x,
                     const hz_solve_params* params, hz_solve_info* infos);
int hz_solve_batched_ex(int nsys, const hz_op* ops, const double* const* b, const double* const* x0,
                        double* const* x, const hz_solve_params* params, hz_solve_info* infos, int strategy);

/* Test hook of hz_solve_batched (process-wide, affects later batched calls):
   timeout_ns bounds every grid-barrier wait of the persistent kernel (<= 0:
   the default, 2 s); leave_block >= 0 makes that block leave the kernel after
   its first barrier, so that the other blocks' waits run out and the call
   returns HZ_ERR_TIMEOUT without hanging the GPU (-1: off). */
int hz_batched_debug(long long timeout_ns, int leave_block);

/* Launch shape of the persistent batched kernel (process-wide, affects later
   batched calls): columns per thread, 1 or 4; 0 (the default) chooses per
   batch: 4 when every nx is a multiple of 4, else 1.  4 with an nx that is
   not a multiple of 4 makes the batched call return HZ_ERR_INVALID.
   Returns HZ_ERR_INVALID for any other value. */
int hz_batched_set_vec(int vec);

/* ---- learned preconditioner stage ----------------------------------------
 * Not in the paper: an extra preconditioner stage inside the flexible solver.
 * After the paper's tridiagonal stage z1 = T^-1 v, the remaining residual
 * e1 = v - D^-1 A z1 is fed to a small 3-D conv net whose output corrects z1:
 *   z = z1 + sigma * NN(e1 / sigma),  sigma = rms(e1).
 * NN: four convolutions 1 -> 16 -> 16 -> 16 -> 1 channels, kernels 3 (k) x
 * 3 (j) x 3 (i), exact-erf GELU after the first three; cross-correlation
 * y[o,p] = b[o] + sum_{c,tap} W[o][c][tap] x[c,p+tap], zero padding in k and
 * j, periodic in i on full fields (zero padding for training crops).  BF16
 * weights and activations, FP32 accumulation; the 16 -> 16 layers on tensor
 * cores.  Parameters: one flat FP32 vector, per layer W[Cout][Cin][3][3][3]
 * (tap order dk, dj, di = -1..1 each, last fastest) then b[Cout];
 * hz_nn_num_params() values.  Training: relative MSE ||y - t||^2 / ||t||^2
 * over the interior of each crop (border points excluded), Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8) on FP32 master weights.  All pointers below are
 * device pointers unless noted.
 */
typedef struct hz_nn_s* hz_nn;
int hz_nn_num_params(void);
const char* hz_nn_last_error(void);
int hz_nn_create(void* stream, hz_nn* out); /* zero parameters */
int hz_nn_destroy(hz_nn nn);
/* params: host or device, hz_nn_num_params() floats; resets the Adam state */
int hz_nn_set_params(hz_nn nn, const float* params);
int hz_nn_get_params(hz_nn nn, float* out /* host or device */);
/* y = NN(x) on an nx x ny x nz field (ny = several crops of seg_ny rows
   stacked along j, or seg_ny = ny); periodic: wrap in i.  zout (may be NULL):
   receives the FP32 pre-activations z1, z2, z3 as [3][n][16]. */
int hz_nn_forward(hz_nn nn, int nx, int ny, int nz, int seg_ny, int periodic, const float* x, float* y, float* zout);
/* gradient of the masked relative MSE of NN(x) against t (border points of
   every crop excluded in i and j); grad: host or device doubles, loss: host */
int hz_nn_gradient(hz_nn nn, int nx, int ny, int nz, int seg_ny, int periodic, int border, const float* x,
                   const float* t, double* grad, double* loss);
/* the gradient of the operator-weighted loss (see hz_nn_train_params.loss) on
   stacked crops (no wrap in i): bands = the crops' six scaled bands
   E,W,N,S,U,D of D^-1 A ([6][nx*ny*nz], host or device floats); border (>= 1)
   excludes the points near each crop's edges in i and j from the residual;
   neighbours outside a crop are absent.  grad: host or device doubles. */
int hz_nn_gradient_op(hz_nn nn, int nx, int ny, int nz, int seg_ny, int border, const float* x, const float* t,
                      const float* bands, double* grad, double* loss);
/* one Adam step on that loss; the gradient is first scaled down to global
   2-norm clip when it is larger (clip <= 0: no clipping).  loss: host, may be NULL */
int hz_nn_train_step(hz_nn nn, int nx, int ny, int nz, int seg_ny, int periodic, int border, const float* x,
                     const float* t, double lr, double clip, double* loss);
/* ncrop crops of cx x cy columns, all levels, from two fields [nz][ny][nx]:
   crop q starts at column (corners[2q], corners[2q+1]) (host ints; i wraps,
   rows outside the grid are zero); outputs [nz][ncrop*cy][cx] (crops stacked
   along j).  The random corners are an input. */
int hz_nn_crops(int nx, int ny, int nz, const float* fa, const float* fb, int ncrop, int cx, int cy,
                const int* corners, float* oa, float* ob, void* stream);
/* checkpoint: FP32 master weights, Adam moments and step (host file) */
int hz_nn_save(hz_nn nn, const char* path);
int hz_nn_load(hz_nn nn, const char* path);
/* ---- storage of the horizontal bands ---------------------------------------
 * The paper's argument for 32-bit numbers (Secs. 1 and 3) is that smaller
 * data moves less.  Carried one step further: the four horizontal bands
 * E, W, N, S of D^-1 A, read by the stencil kernels twice per inner BiCGStab
 * iteration, can be stored in 16 bits (BF16: 8 significant bits, the FP32
 * range; FP16: 11 significant bits, values below 6.1e-5 subnormal), widened
 * to FP32 for the arithmetic.  The vertical part T (the U and D bands and the
 * Thomas factors) stays FP32: its rows sum to nearly zero, and 16-bit
 * rounding would change the near-singular columns.  The FP64 outer residual
 * keeps the exact FP64 A, so the refinement loop corrects what the rounding
 * changes (at the cost of the inner solves' convergence).  The format applies
 * to the FP32 BiCGStab solver with T^-1 (mixed mode and HZ_MODE_PAPER_MP) and
 * to hz_matvec and hz_precond_matvec in HZ_PREC_FP32; FGMRES, tri-SOR, the
 * batched solver and hz_nn_make_pair read the FP32 bands.  The 16-bit copies
 * (8 bytes per point) are made on the first call and redone by
 * hz_op_update.  Rounding: to nearest even, BF16 from the FP32 value, FP16
 * from the FP64 value. */
#define HZ_BANDS_FP32 0
#define HZ_BANDS_BF16 1
#define HZ_BANDS_FP16 2
int hz_op_set_band_format(hz_op op, int fmt);
int hz_op_get_band_format(hz_op op, int* fmt);

/* attach a network to an operator for params->precond = HZ_PRE_TRI_NN (NULL detaches) */
int hz_op_set_nn(hz_op op, hz_nn nn);
/* Training pair of an iterate x_k with exact solution x_star (all FP64, n):
   r = D^-1 (b - A x_k), e = x_star - x_k, z1 = T^-1 r, e1 = r - D^-1 A z1;
   in = e1 / sigma, target = (e - z1) / sigma, sigma = rms(e1) (host out). */
int hz_nn_make_pair(hz_op op, const double* b, const double* xk, const double* x_star, float* in, float* target,
                    double* sigma);

/* Training of the learned stage on one system (not in the paper: the stage is
 * an extra preconditioner of the flexible solver).  For the operator op and
 * right-hand side b (device, n doubles):
 *   1. x* = the FP64 solution to xstar_tol (hz_solve, HZ_MODE_FP64);
 *   2. for each k in iterates: x_k = the mixed solver's iterate after one
 *      refinement step of k inner iterations from x = 0, and its training pair
 *      (stage input, target) from hz_nn_make_pair;
 *   3. steps Adam steps (hz_nn_train_step, with clip), each on batch crops of
 *      one pair: (crop + 8) x (crop + 8) columns and all levels (a halo of 4
 *      columns, the receptive field of the four 3x3x3 layers, is excluded from
 *      the loss), stacked along j.  The pair and the crop corners (i0 uniform
 *      over the row, j0 uniform over [0, ny - crop)) are drawn from a
 *      counter-based generator: SplitMix64 (Steele, Lea and Flood 2014) keyed
 *      by (seed, stream, draw number), so a call is reproducible.
 * The network's Adam state carries over from call to call: train on many
 * systems by calling once per system (each operator can be created just
 * before and destroyed after its call), with its own stream value.
 * Requires crop + 8 <= nx and crop < ny.  losses: host array of steps values
 * (the loss of each step, before its update), may be NULL.  Device memory for
 * x*, the iterates and the pairs is allocated for the call and freed after it.
 * Errors: HZ_ERR_INVALID (arguments), the errors of the calls above. */
typedef struct {
  int steps;          /* Adam steps on this system's pairs (default 40) */
  int batch;          /* crops per step (default 16) */
  int crop;           /* interior width of a crop in columns (default 64) */
  int n_iterates;     /* 1..16 entries of iterates used (default 6) */
  int iterates[16];   /* inner iterations k of the iterates x_k (default 1, 2, 4, 8, 16, 32) */
  double xstar_tol;   /* tolerance of the FP64 solve for x* (default 1e-11) */
  double lr;          /* Adam learning rate (default 3e-4) */
  double clip;        /* global gradient 2-norm clip (default 1; <= 0: none) */
  unsigned long long seed;    /* random draws: (seed, stream) select the counter stream */
  unsigned long long stream;
  int loss;           /* 1 (default): operator-weighted, ||D^-1 A (y - t)||^2 / ||D^-1 A t||^2 over the crop
                         interior less one more column (with t the pair's target, D^-1 A t is the stage
                         input: the squared relative residual left after the stage); 0: the relative MSE
                         ||y - t||^2 / ||t||^2 of hz_nn_train_step */
} hz_nn_train_params;
void hz_nn_train_defaults(hz_nn_train_params* p);
int hz_nn_train(hz_nn nn, hz_op op, const double* b, const hz_nn_train_params* p, double* losses);

/* Inner recursive residual history of the last solve with record_history=1:
   copies up to cap values into hist (host) and returns how many. */
int hz_get_history(hz_op op, double* hist, int cap);

/*
 * Autotuner for the column kernels (not in the paper: a launch-shape search).
 * The Thomas kernels (k_pre_p, k_pre_s) and the stencil kernels (k_mv) come
 * in variants: vec columns per thread (vector loads; vec must divide nx) and
 * depth levels per software-pipelined batch; a Thomas variant also fixes
 * where the forward sweep waits for the back sweep (the output vector, shared
 * memory, or the output vector stored with the L2 evict-last priority while
 * the streamed arrays are evict-first, or a warp-specialised kernel staging
 * its inputs by bulk copies); Thomas and stencil variants may cap the
 * resident blocks per SM.  All variants of a kernel compute the same values; dot partial sums
 * follow the launch shape.  hz_op_autotune times every
 * valid variant on the operator's own arrays (3 launches each, CUDA events on
 * the operator's stream) and keeps the fastest, or the lowest-numbered variant
 * within 2% of it (a stable choice: the dot products' rounding, hence the
 * iteration count, follows the variant); flags bit 0 also tunes the
 * FP64 kernels (allocating the FP64 work vectors); flags bit 1 also tunes the
 * tri-SOR kernels (for nx even; allocating their colour-compact copies of the
 * bands), in FP32 and, with bit 0, FP64.  If the environment
 * variable HZ_AUTOTUNE_CACHE names a file, results are appended to it (one
 * line per device, grid, precision and kernel kind) and read back by
 * hz_op_create for operators of the same grid.  Variant ids: 0 .. count-1 of
 * the tables in the library; hz_op_set_variants takes -1 for "unchanged".
 * The work vectors are overwritten; call between solves.
 */
int hz_op_autotune(hz_op op, int flags);
/* tri-SOR kernel variants: kind 0 = colour pass, 1 = matvec, 2 = first pass
   (vector update fused with the first red pass); each is a (columns per
   thread, levels per batch, blocks per SM) shape, some with L2 priorities
   (once-read arrays evict-first, the parked forward sweep evict-last).  Count per prec (HZ_PREC_*) and kind (0 for an
   invalid pair); get/set the operator's choice (set: HZ_ERR_INVALID for an id
   out of range).  Every variant computes the same columns the same way; the
   matvec's dot partial sums follow the shape. */
int hz_sor_variant_count(int prec, int kind);
int hz_op_get_sor_variant(hz_op op, int prec, int kind, int* id);
int hz_op_set_sor_variant(hz_op op, int prec, int kind, int id);
int hz_op_get_variants(hz_op op, int* pre32, int* mv32, int* pre64, int* mv64);
int hz_op_set_variants(hz_op op, int pre32, int mv32, int pre64, int mv64);

/*
 * Per-kernel profile.  While enabled, solves run the host-driven loop with a
 * pair of CUDA events on the operator's stream around every kernel launch
 * (slower: each launch is waited for), and hz_profile_read returns, for
 * kernel kid, the launches, their summed device time in ms and their summed
 * algorithmic bytes (each array element read or written once per launch).
 * Enabling (or disabling) resets the counters.  hz_op_update is profiled too.
 */
/* ids: 0 k_setup, 1 k_residual, 2 k_pre_p, 3 k_mv_v, 4 k_pre_s, 5 k_mv_t, 6 k_upd,
   and for HZ_PRE_TRISOR: 7 k_sor_first (vector update + first red pass),
   8 k_sor_pass (colour passes), 9 k_mv_rb (Ahat matvec + dots), 10 k_rb_copy
   (natural <-> colour-compact order around each refinement step) */
#define HZ_NUM_KERNELS 11
int hz_profile_enable(hz_op op, int on);
int hz_profile_read(hz_op op, int kid, long long* launches, double* ms, double* bytes);
const char* hz_kernel_name(int kid);

/* ---- kernel-level entry points (the building blocks of the solve, exposed for testing) ---- */

/* y = D^-1 A x (unit diagonal, six scaled bands) in the given precision.
   x, y: device arrays of n floats (HZ_PREC_FP32) or doubles (HZ_PREC_FP64). */
int hz_matvec(hz_op op, int prec, const void* x, void* y);

/* z = T^-1 r, T = per-column tridiagonal part of D^-1 A (Sec. 2), using the
   pre-computed factors.  r, z: device arrays in the given precision; may not alias. */
int hz_precond_apply(hz_op op, int prec, const void* r, void* z);

/* v = D^-1 A (T^-1 p) as the solver forms it: ph = T^-1 p, then
   v = p + H ph with H the four horizontal bands (T ph = p).  p, ph, v: device. */
int hz_precond_matvec(hz_op op, int prec, const void* p, void* ph, void* v);

/* z = C r with C the tri-SOR preconditioner of Sec. 2: `sweeps` (1..64)
   red-black sweeps x_n = (1-w) x_(n-1) + w T^-1 (r - L x_n - U x_(n-1)) from
   x_0 = 0, w = omega in (0, 2), in the given precision; the same kernels as
   the solver (which work in colour-compact column order: r is gathered into
   it and z scattered back).  r, z: device arrays in natural order; may not
   alias.  Needs nx even (HZ_ERR_UNSUPPORTED).  Overwrites the operator's
   inner work vectors of that precision: call between solves. */
int hz_trisor_apply(hz_op op, int prec, int sweeps, double omega, const void* r, void* z);

/* True FP64 residual (Sec. 3): r = b - A x with the unscaled bands.
   b, x: device doubles; r: device doubles or NULL; rnorm, bnorm: host outputs (may be NULL). */
int hz_residual(hz_op op, const double* b, const double* x, double* r, double* rnorm, double* bnorm);

/* Deterministic dot product sum_i x_i y_i of device arrays (float or double
   by prec; FP64 accumulation across threads and blocks).  out: host. */
int hz_dot(int prec, int64_t n, const void* x, const void* y, void* stream, double* out);

/*
 * hz_dot_noalloc -- the deterministic dot product of hz_dot for callers that
 * cannot allocate device memory.  The paper has no counterpart: it is a
 * deployment aid.  hz_dot allocates its scratch with cudaMalloc on its first
 * call on a device; code that must not allocate (inside a fixed memory pool,
 * under an allocator owned by another framework, or under a no-allocation
 * rule after start-up) cannot use it.  This entry point allocates nothing:
 * its scratch is a static device array of HZ_DOT_NOALLOC_SLOTS partial sums
 * plus a ticket word (32 KiB, held by every GPU that loads the library until
 * the process exits), and it calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *   prec: HZ_PREC_FP32 or HZ_PREC_FP64; x, y: device arrays of n elements;
 *   out: DEVICE pointer to one double that receives sum_i x_i y_i (FP64
 *   accumulation, same kernel and order as hz_dot for the same launch shape);
 *   stream: the stream to order the work on.  The call does not wait.
 * Limits: n >= 0; at most HZ_DOT_NOALLOC_SLOTS blocks are launched (grid-
 * stride), so any n fits the scratch.  Invalid arguments return
 * HZ_ERR_INVALID.
 * Set-up: the first call on each device looks up the array's device address
 * (with that device current); make that first call before any stream capture.
 * Sharing: every call uses the same array and leaves its contents behind;
 * each call zeroes the ticket it needs first.  Calls that overlap on the GPU
 * (concurrent streams, or several host threads) race on the array and give
 * wrong results: serialise them.
 */
#define HZ_DOT_NOALLOC_SLOTS 4064
int hz_dot_noalloc(int prec, int64_t n, const void* x, const void* y, void* stream, double* out);

/* Copy the operator's derived data to device memory dst:
   what = 0: scaled bands [6][n] (E,W,N,S,U,D) in prec;
   what = 1: Thomas factors [3][n] (m, l, c') in prec, where the forward sweep
             is y_k = m_k p_k - l_k y_(k-1) and the back sweep z_k = y_k - c'_k z_(k+1);
   what = 2: the 16-bit horizontal bands [4][n] (E,W,N,S; the bit patterns) of an
             operator whose band format is BF16 or FP16 (prec ignored; else HZ_ERR_INVALID). */
int hz_op_export(hz_op op, int what, int prec, void* dst);

#ifdef __cplusplus
}
#endif
#endif /* HZ_H_ */
