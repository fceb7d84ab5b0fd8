"""CPU oracle for the Helmholtz solve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (``paper_1811_03852_gb300``)
never imports, links or runs it, and the two share no code: the oracle is
plain C (``hz_oracle.c``, serial; an OpenMP build of the same source, with
the same results, times it on all host cores) plus the NumPy conv-net
reference in ``nn.py``, written from Maynard & Walters (arXiv:1811.03852) and
from the textbook definitions they cite.  Inputs come from the separate ``gen``
package, which holds no solver arithmetic.

Every routine is pinned by ``tests/test_oracle_*.py`` against something other
than itself (dense LAPACK solves, banded solves, closed forms, brute force,
finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hz_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhz_oracle.so")
_LIB_OMP = os.path.join(_BUILD, "libhz_oracle_omp.so")
_lock = threading.Lock()
_libs = {}
_use_omp = False

MODE_FP64 = 0
MODE_MIXED = 1
MODE_PAPER_MP = 2

# -ffp-contract=off: every a*b+c is two rounded operations as written, on x86
# and Arm alike (gcc would otherwise fuse them where the target has an FMA)
_CFLAGS = ["-O3", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle, serial (the tests' oracle) and with OpenMP (for timing it on
    all host cores; same source, same bits), if missing or stale.  Returns the serial library."""
    os.makedirs(_BUILD, exist_ok=True)
    for lib, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(_SRC):
            continue
        tmp = f"{lib}.{os.getpid()}.tmp"
        subprocess.run(["gcc"] + _CFLAGS + extra + ["-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, lib)
    return _LIB


def use_openmp(on: bool = True, threads: int | None = None) -> int:
    """Route every oracle call through the OpenMP build (on=True) or the serial one.
    threads: OpenMP threads (None: the runtime's default, all host cores).  The two
    builds compute the same values bit for bit (fixed-chunk sums); this only changes
    how long the oracle takes.  Returns the number of threads in use."""
    global _use_omp
    _use_omp = bool(on)
    L = _load()
    if on and threads:
        L.or_set_threads(int(threads))
    return int(L.or_threads())


def _load():
    with _lock:
        key = "omp" if _use_omp else "serial"
        if key not in _libs:
            build()
            lib = ctypes.CDLL(_LIB_OMP if _use_omp else _LIB)
            i32, dbl, pv, i64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64
            lib.or_matvec.argtypes = [i32, i32, i32, pv, pv, pv]
            lib.or_matvec.restype = None
            lib.or_residual.argtypes = [i32, i32, i32, pv, pv, pv, pv]
            lib.or_residual.restype = dbl
            lib.or_scale.argtypes = [i32, i32, i32, pv, pv]
            lib.or_scale.restype = None
            lib.or_matvec_hat.argtypes = [i32, i32, i32, pv, pv, pv]
            lib.or_matvec_hat.restype = None
            lib.or_tridiag_solve.argtypes = [i32, pv, pv, pv, pv, pv, pv]
            lib.or_tridiag_solve.restype = None
            lib.or_apply_Tinv.argtypes = [i32, i32, i32, pv, pv, pv]
            lib.or_apply_Tinv.restype = None
            lib.or_bicgstab.argtypes = [i32, i32, i32, pv, pv, pv, dbl, i32, i32, pv, pv]
            lib.or_bicgstab.restype = None
            lib.or_bicgstab_f32.argtypes = [i32, i32, i32, pv, pv, pv, dbl, i32, i32, pv, pv]
            lib.or_bicgstab_f32.restype = None
            lib.or_bicgstab_mp.argtypes = [i32, i32, i32, pv, pv, pv, dbl, i32, i32, pv, pv]
            lib.or_bicgstab_mp.restype = None
            lib.or_solve.argtypes = [i32, i32, i32, pv, pv, pv, i32, dbl, dbl, i32, i32, i32, pv, pv, pv]
            lib.or_solve.restype = None
            lib.or_dot.argtypes = [i64, pv, pv]
            lib.or_dot.restype = dbl
            lib.or_set_threads.argtypes = [i32]
            lib.or_set_threads.restype = None
            lib.or_threads.argtypes = []
            lib.or_threads.restype = i32
            _libs[key] = lib
        return _libs[key]


def _c(a, dtype=np.float64):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _p(a):
    return a.ctypes.data


def _dims(x):
    nz, ny, nx = x.shape[-3:]
    return nx, ny, nz


def matvec(A, x):
    """y = A x (unscaled 7-band operator, Sec. 1 eq. LinearSys / Sec. 2 Helmholtz)."""
    A, x = _c(A), _c(x)
    nx, ny, nz = _dims(x)
    y = np.empty_like(x)
    _load().or_matvec(nx, ny, nz, _p(A), _p(x), _p(y))
    return y


def residual(A, b, x):
    """(r = b - A x, ||r||_2)."""
    A, b, x = _c(A), _c(b), _c(x)
    nx, ny, nz = _dims(x)
    r = np.empty_like(x)
    nrm = _load().or_residual(nx, ny, nz, _p(A), _p(b), _p(x), _p(r))
    return r, nrm


def scale(A):
    """Ahat = D^-1 A off-diagonal bands (6, nz, ny, nx), order E,W,N,S,U,D."""
    A = _c(A)
    nz, ny, nx = A.shape[1:]
    Ah = np.empty((6, nz, ny, nx))
    _load().or_scale(nx, ny, nz, _p(A), _p(Ah))
    return Ah


def matvec_hat(Ah, x):
    """y = Ahat x with unit diagonal."""
    Ah, x = _c(Ah), _c(x)
    nx, ny, nz = _dims(x)
    y = np.empty_like(x)
    _load().or_matvec_hat(nx, ny, nz, _p(Ah), _p(x), _p(y))
    return y


def tridiag_solve(lo, di, up, r):
    """Solve one tridiagonal system (Thomas algorithm, factors recomputed)."""
    lo, di, up, r = (_c(v) for v in (lo, di, up, r))
    m = r.size
    x = np.empty(m)
    wk = np.empty(2 * m)
    _load().or_tridiag_solve(m, _p(lo), _p(di), _p(up), _p(r), _p(x), _p(wk))
    return x


def apply_Tinv(Ah, r):
    """z = T^-1 r, T = per-column tridiagonal part (D band, 1, U band) of Ahat."""
    Ah, r = _c(Ah), _c(r)
    nx, ny, nz = _dims(r)
    z = np.empty_like(r)
    _load().or_apply_Tinv(nx, ny, nz, _p(Ah), _p(r), _p(z))
    return z


def bicgstab(Ah, bh, x0=None, eta=1e-8, maxit=1000, restart=150, fp32=False, history=False, x64=False):
    """Right-preconditioned BiCGStab with C = T^-1 on Ahat y = bh.

    Returns (x, info dict[, hist]).  With fp32=True every vector and
    coefficient is a float and dots accumulate in double; with x64=True as
    well, the iterate x is kept in double (the paper's mixed-precision
    solver, Sec. 3) and returned as float64.
    """
    nz, ny, nx = bh.shape
    dt = np.float32 if fp32 else np.float64
    Ah_ = _c(Ah, dt)
    bh_ = _c(bh, dt)
    xdt = np.float64 if (x64 or not fp32) else np.float32
    x = np.zeros(bh_.shape, dtype=xdt) if x0 is None else _c(x0, xdt).copy()
    hist = np.full(maxit, np.nan)
    out = np.zeros(4)
    fn = (_load().or_bicgstab_mp if x64 else _load().or_bicgstab_f32) if fp32 else _load().or_bicgstab
    fn(nx, ny, nz, _p(Ah_), _p(bh_), _p(x), eta, maxit, restart, _p(hist), _p(out))
    info = dict(iters=int(out[0]), restarts=int(out[1]), relres=float(out[2]), status=int(out[3]))
    if history:
        return x, info, hist[: info["iters"]]
    return x, info


def solve(A, b, x0=None, mode=MODE_MIXED, tol=1e-8, eta=1e-4, max_outer=20, max_inner=2000, restart=150,
          history=False, inner_bands=None):
    """Outer loop on the true FP64 residual with FP64 (mode 0) or FP32 (mode 1) inner BiCGStab;
    mode 2 is the paper's mixed-precision solver (one solve, x in FP64, the rest FP32, no refinement).
    inner_bands: the FP32 inner operator (6, nz, ny, nx) of modes 1 and 2 instead of float(Ahat),
    e.g. round_hbands(scale(A), fmt).

    Returns (x, info dict[, outer history of R]).
    """
    A, b = _c(A), _c(b)
    nx, ny, nz = _dims(b)
    x = np.zeros_like(b) if x0 is None else _c(x0).copy()
    hist = np.full(max_outer + 1, np.nan)
    out = np.zeros(5)
    ib = None if inner_bands is None else _c(inner_bands, np.float32)
    _load().or_solve(nx, ny, nz, _p(A), _p(b), _p(x), mode, tol, eta, max_outer, max_inner, restart, _p(hist),
                     _p(out), None if ib is None else _p(ib))
    info = dict(outer=int(out[0]), inner=int(out[1]), R=float(out[2]), status=int(out[3]), restarts=int(out[4]))
    if history:
        return x, info, hist[: info["outer"] + 1]
    return x, info


def dot(a, b):
    a, b = _c(a).ravel(), _c(b).ravel()
    return _load().or_dot(a.size, _p(a), _p(b))


def apply_trisor(Ah, r, sweeps=3, omega=1.5):
    """z = C r, C = `sweeps` red-black tri-SOR sweeps from zero (Sec. 2 fixed point)."""
    Ah, r = _c(Ah), _c(r)
    nx, ny, nz = _dims(r)
    z = np.empty_like(r)
    L = _load()
    if not getattr(L, "_sor_sig", False):
        L.or_apply_trisor.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 3 + [ctypes.c_int, ctypes.c_double]
        L.or_apply_trisor.restype = None
        L.or_set_precond.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.or_set_precond.restype = None
        L._sor_sig = True
    L.or_apply_trisor(nx, ny, nz, _p(Ah), _p(r), _p(z), sweeps, omega)
    return z


def set_precond(kind, sweeps=3, omega=1.5):
    """Preconditioner of bicgstab()/solve(): kind 0 = T^-1 (default), 1 = tri-SOR(sweeps, omega)."""
    apply_trisor  # noqa: B018  (ensures signatures below)
    L = _load()
    L.or_set_precond.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
    L.or_set_precond.restype = None
    L.or_set_precond(kind, sweeps, omega)


# ---- 16-bit storage of the horizontal bands ---------------------------------------
def round_bf16(x):
    """x rounded to bfloat16 (1 sign, 8 exponent, 7 fraction bits; the FP32 exponent range), to
    nearest with ties to even, from the FP32 rounding of x; returned as float64 values.
    Written from the format: keep the top 16 bits of the FP32 pattern, adding half of the last
    kept place (less one) plus the kept place's lowest bit before truncating."""
    f = np.ascontiguousarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_fp16(x):
    """x rounded to IEEE binary16 (to nearest, ties to even, subnormals below 2^-14), as float64."""
    return np.ascontiguousarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def bits16(x, fmt):
    """The 16-bit patterns of values already rounded to the format (1 = BF16, 2 = FP16)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if fmt == 1:
        return (x.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
    return x.astype(np.float16).view(np.uint16)


def round_hbands(Ah, fmt):
    """Ahat with its horizontal bands E, W, N, S (rows 0..3) rounded to BF16 (fmt 1) or FP16
    (fmt 2) and the vertical bands U, D unchanged."""
    out = np.array(Ah, dtype=np.float64, copy=True)
    out[:4] = round_bf16(out[:4]) if fmt == 1 else round_fp16(out[:4])
    return out

