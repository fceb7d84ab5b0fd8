"""Seeded synthetic Helmholtz systems (input generator shared by the oracle and the GPU path).

This package only synthesises inputs: the seven coefficient bands of the
ENDGame-like pressure-correction operator and a smooth right-hand side
(Maynard & Walters, Sec. 2: a 7-band, nonsymmetric, variable-coefficient
matrix on a lon-lat grid with vertical levels).  It contains none of the
solver's arithmetic.  The work is done by ``hzgen.c`` (OpenMP), compiled on
first use with gcc into ``gen/_build/``.

Recipe (one reading per choice):
  * grid nx x ny x nz, dlambda = 2 pi/nx, dphi = pi/ny, phi_j = -pi/2 + (j+1/2) dphi;
  * dz_k = 20 + 1980 (k/(nz-1))^2 metres, converted by ``z_unit``
    ("radius": Earth radii, the default; "m": metres, the hard family);
  * weights E,W = 1/(cos phi dlambda)^2, N,S = 1/dphi^2, U,D = 1/dz_k^2, each times
    exp(0.1 xi), xi ~ N(0,1) iid per point and band; zero flux across the
    pole rows and through the top and bottom;
  * off-diagonal a_b = -w_b (1 - 0.05 s_b), s = +1 for E,N,U and -1 for W,S,D;
  * diagonal a_C = -sum_b a_b + c, c = 1e-3 max w;
  * b = 16 smooth separable modes (unit RMS) + 0.01 N(0,1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hzgen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhzgen.so")
_lock = threading.Lock()
_lib = None

BANDS = ("C", "E", "W", "N", "S", "U", "D")
EARTH_RADIUS_M = 6.371e6


def build(force: bool = False) -> str:
    """Compile libhzgen.so (gcc, OpenMP) if it is missing or older than its source."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = f"{_LIB}.{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i32, dbl, pd = ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.hzgen_operator.argtypes = [i32, i32, i32, u64, dbl, dbl, dbl, dbl, pd]
            lib.hzgen_operator.restype = i32
            lib.hzgen_rhs.argtypes = [i32, i32, i32, u64, dbl, pd]
            lib.hzgen_rhs.restype = i32
            lib.hzgen_normals.argtypes = [u64, u64, ctypes.c_int64, pd]
            lib.hzgen_normals.restype = None
            lib.hzgen_uniform.argtypes = [u64, u64, u64]
            lib.hzgen_uniform.restype = dbl
            lib.hzgen_normal.argtypes = [u64, u64, u64]
            lib.hzgen_normal.restype = dbl
            lib.hzgen_bits.argtypes = [u64, u64, u64]
            lib.hzgen_bits.restype = u64
            _lib = lib
    return _lib


def z_scale(z_unit: str) -> float:
    if z_unit in ("radius", "r", "earth"):
        return 1.0 / EARTH_RADIUS_M
    if z_unit in ("m", "metre", "meter", "metres"):
        return 1.0
    raise ValueError(f"unknown z_unit {z_unit!r}")


def _ptr_of(buf, n, dtype=np.float64):
    if buf is None:
        arr = np.empty(n, dtype=dtype)
        return arr, arr.ctypes.data
    if isinstance(buf, np.ndarray):
        assert buf.dtype == dtype and buf.size == n and buf.flags.c_contiguous
        return buf, buf.ctypes.data
    # torch tensor (e.g. pinned host memory): duck-typed
    assert buf.numel() == n and buf.is_contiguous() and not buf.is_cuda
    return buf, buf.data_ptr()


def make_operator(nx, ny, nz, seed, z_unit="radius", sigma=0.1, skew=0.05, shift_frac=1e-3, out=None):
    """Coefficient bands, shape (7, nz, ny, nx) float64, band order C,E,W,N,S,U,D.

    ``out`` may be a preallocated contiguous float64 buffer (numpy or CPU torch) of 7*n values.
    """
    n = nx * ny * nz
    arr, p = _ptr_of(out, 7 * n)
    rc = _load().hzgen_operator(nx, ny, nz, seed, z_scale(z_unit), sigma, skew, shift_frac, p)
    if rc != 0:
        raise ValueError(f"hzgen_operator failed ({rc})")
    return arr.reshape(7, nz, ny, nx) if isinstance(arr, np.ndarray) else arr


def make_rhs(nx, ny, nz, seed, noise_frac=0.01, out=None):
    """Right-hand side, shape (nz, ny, nx) float64."""
    n = nx * ny * nz
    arr, p = _ptr_of(out, n)
    rc = _load().hzgen_rhs(nx, ny, nz, seed, noise_frac, p)
    if rc != 0:
        raise ValueError(f"hzgen_rhs failed ({rc})")
    return arr.reshape(nz, ny, nx) if isinstance(arr, np.ndarray) else arr


def make_system(nx, ny, nz, seed_coef, seed_rhs, z_unit="radius"):
    """(coeffs (7,nz,ny,nx), b (nz,ny,nx)) in float64."""
    return make_operator(nx, ny, nz, seed_coef, z_unit), make_rhs(nx, ny, nz, seed_rhs)


def normals(seed, stream, count):
    """count seeded N(0,1) values (test vectors), float64."""
    out = np.empty(count, dtype=np.float64)
    _load().hzgen_normals(seed, stream, count, out.ctypes.data)
    return out


def uniform(seed, stream, ctr):
    return _load().hzgen_uniform(seed, stream, ctr)


# ---- named workloads (grid, coefficient seed, rhs seed) -------------------------------
WORKLOADS = {
    "plain96": dict(nx=96, ny=72, nz=20, seed_coef=1, seed_rhs=2),
    "mixed640": dict(nx=640, ny=480, nz=70, seed_coef=11, seed_rhs=12),
    "n1280": dict(nx=2560, ny=1920, nz=70, seed_coef=21, seed_rhs=22),
}

BATCHED_GRIDS = ((192, 144), (320, 240), (640, 480))


def batched_spec(i):
    """System i of the 32-system uneven batch: grid cycles through 192x144, 320x240, 640x480 (70 levels)."""
    gx, gy = BATCHED_GRIDS[i % 3]
    return dict(nx=gx, ny=gy, nz=70, seed_coef=1000 + 2 * i, seed_rhs=1001 + 2 * i)
