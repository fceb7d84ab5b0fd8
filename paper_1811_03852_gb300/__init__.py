"""GB300 (sm_103a) mixed-precision Helmholtz solver -- thin Python binding of libhz.so.

The solver is the method of Maynard & Walters, "Precision of the ENDGame"
(arXiv:1811.03852): post-conditioned BiCGStab on D^-1 A with the per-column
vertical tridiagonal preconditioner (Sec. 2), FP32 inner iterations and FP64
global sums (Secs. 3-4), wrapped in an outer FP64 iterative-refinement loop
on the true residual R = ||b - A x|| / ||b||.

Every step of the solve runs in the CUDA library; this module only marshals
arguments through ctypes (names match include/hz.h).  PyTorch is used for
device memory and streams.  There is no CPU fallback: importing the package
on a machine without the built library, or calling a compute entry point
without a GPU, raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

_PKG = os.path.dirname(os.path.abspath(__file__))

HZ_OK = 0
HZ_ERR_INVALID = 1
HZ_ERR_CUDA = 2
HZ_ERR_OOM = 3
HZ_ERR_NOT_CONVERGED = 4
HZ_ERR_BREAKDOWN = 5
HZ_ERR_NONFINITE = 6
HZ_ERR_TIMEOUT = 7
HZ_ERR_UNSUPPORTED = 8

HZ_BATCH_AUTO, HZ_BATCH_PERSISTENT, HZ_BATCH_SEQUENTIAL = 0, 1, 2
HZ_MODE_FP64 = 0
HZ_MODE_MIXED_IR = 1
HZ_MODE_PAPER_MP = 2
HZ_MODE_PAPER_DP = 3
HZ_PREC_FP64 = 0
HZ_PREC_FP32 = 1
HZ_PRE_TRI = 0
HZ_PRE_TRI_NN = 1
HZ_PRE_TRISOR = 2
HZ_BANDS_FP32, HZ_BANDS_BF16, HZ_BANDS_FP16 = 0, 1, 2
HZ_KRYLOV_BICGSTAB = 0
HZ_KRYLOV_FGMRES = 1
NUM_KERNELS = 11


class hz_solve_params(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("inner_tol", ctypes.c_double),
        ("mode", ctypes.c_int),
        ("precond", ctypes.c_int),
        ("krylov", ctypes.c_int),
        ("max_outer", ctypes.c_int),
        ("max_inner", ctypes.c_int),
        ("restart", ctypes.c_int),
        ("fgmres_m", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("record_history", ctypes.c_int),
        ("sor_sweeps", ctypes.c_int),
        ("sor_omega", ctypes.c_double),
        ("dot_fp32", ctypes.c_int),
        ("nn_window", ctypes.c_int),
        ("nn_factor", ctypes.c_double),
    ]


class hz_solve_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("outer_iters", ctypes.c_int),
        ("inner_iters", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("fallbacks", ctypes.c_int),
        ("fp64_retries", ctypes.c_int),
        ("true_rel_residual", ctypes.c_double),
        ("scaled_rel_residual", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("kernel_launches", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhz.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libhz.so not built at {path}; run paper_1811_03852_gb300._build.build()")
    L = ctypes.CDLL(path)
    i32, i64, dbl, pv = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "hz_version": (i32, []),
        "hz_status_str": (ctypes.c_char_p, [i32]),
        "hz_last_error": (ctypes.c_char_p, []),
        "hz_default_params": (None, [P(hz_solve_params)]),
        "hz_op_create": (i32, [i32, i32, i32, pv, pv, P(pv)]),
        "hz_op_update": (i32, [pv, pv]),
        "hz_op_destroy": (i32, [pv]),
        "hz_op_dims": (i32, [pv, P(i32), P(i32), P(i32)]),
        "hz_solve": (i32, [pv, pv, pv, pv, P(hz_solve_params), P(hz_solve_info)]),
        "hz_solve_batched": (i32, [i32, P(pv), P(pv), P(pv), P(pv), P(hz_solve_params), P(hz_solve_info)]),
        "hz_solve_batched_ex": (i32, [i32, P(pv), P(pv), P(pv), P(pv), P(hz_solve_params), P(hz_solve_info), i32]),
        "hz_get_history": (i32, [pv, pv, i32]),
        "hz_matvec": (i32, [pv, i32, pv, pv]),
        "hz_precond_apply": (i32, [pv, i32, pv, pv]),
        "hz_trisor_apply": (i32, [pv, i32, i32, ctypes.c_double, pv, pv]),
        "hz_sor_variant_count": (i32, [i32, i32]),
        "hz_op_get_sor_variant": (i32, [pv, i32, i32, ctypes.POINTER(i32)]),
        "hz_op_set_sor_variant": (i32, [pv, i32, i32, i32]),
        "hz_precond_matvec": (i32, [pv, i32, pv, pv, pv]),
        "hz_residual": (i32, [pv, pv, pv, pv, P(dbl), P(dbl)]),
        "hz_dot": (i32, [i32, i64, pv, pv, pv, P(dbl)]),
        "hz_op_export": (i32, [pv, i32, i32, pv]),
        "hz_dot_noalloc": (i32, [i32, i64, pv, pv, pv, pv]),
        "hz_batched_debug": (i32, [ctypes.c_longlong, i32]),
        "hz_batched_set_vec": (i32, [i32]),
        "hz_op_autotune": (i32, [pv, i32]),
        "hz_op_get_variants": (i32, [pv, P(i32), P(i32), P(i32), P(i32)]),
        "hz_op_set_variants": (i32, [pv, i32, i32, i32, i32]),
        "hz_profile_enable": (i32, [pv, i32]),
        "hz_profile_read": (i32, [pv, i32, P(ctypes.c_longlong), P(dbl), P(dbl)]),
        "hz_kernel_name": (ctypes.c_char_p, [i32]),
        "hz_op_set_band_format": (i32, [pv, i32]),
        "hz_op_get_band_format": (i32, [pv, P(i32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class HzError(RuntimeError):
    def __init__(self, status, where=""):
        L = load()
        msg = L.hz_status_str(status).decode()
        last = L.hz_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}){' -- ' + last if last else ''}")
        self.status = status


def _check(st, where):
    if st != HZ_OK:
        raise HzError(st, where)


def _ptr(a):
    """Raw pointer of a torch tensor (device or host) or numpy array (host); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def default_params(**kw) -> hz_solve_params:
    p = hz_solve_params()
    load().hz_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class Operator:
    """A Helmholtz operator on the GPU (``hz_op``).

    coeffs: float64 array/tensor of shape (7, nz, ny, nx) (bands C,E,W,N,S,U,D),
    host (numpy / CPU tensor) or CUDA tensor.
    """

    def __init__(self, coeffs, stream=None):
        L = load()
        shape = tuple(coeffs.shape)
        if len(shape) != 4 or shape[0] != 7:
            raise ValueError("coeffs must have shape (7, nz, ny, nx)")
        _, nz, ny, nx = shape
        self.nx, self.ny, self.nz = nx, ny, nz
        self.n = nx * ny * nz
        self._h = ctypes.c_void_p()
        st = L.hz_op_create(nx, ny, nz, _ptr(coeffs), _stream_ptr(stream), ctypes.byref(self._h))
        _check(st, "hz_op_create")

    @property
    def handle(self):
        return self._h

    def update(self, coeffs):
        _check(load().hz_op_update(self._h, _ptr(coeffs)), "hz_op_update")

    def close(self):
        if self._h:
            load().hz_op_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- solve -----------------------------------------------------------------
    def solve(self, b, x, x0=None, params=None, raise_on_error=True, **kw):
        """x <- solution of A x = b.  Returns an hz_solve_info as a dict."""
        p = params if params is not None else default_params(**kw)
        info = hz_solve_info()
        st = load().hz_solve(self._h, _ptr(b), _ptr(x0), _ptr(x), ctypes.byref(p), ctypes.byref(info))
        d = info.as_dict()
        d["status"] = st
        if raise_on_error and st not in (HZ_OK,):
            raise HzError(st, f"hz_solve {d}")
        return d

    def history(self, cap=100000):
        buf = np.zeros(cap)
        n = load().hz_get_history(self._h, buf.ctypes.data, cap)
        return buf[: max(n, 0)]

    # ---- building blocks ---------------------------------------------------------
    def matvec(self, x, y, prec):
        _check(load().hz_matvec(self._h, prec, _ptr(x), _ptr(y)), "hz_matvec")

    def precond_apply(self, r, z, prec):
        _check(load().hz_precond_apply(self._h, prec, _ptr(r), _ptr(z)), "hz_precond_apply")

    def trisor_apply(self, r, z, prec, sweeps=3, omega=1.5):
        """z = C r, C = `sweeps` red-black tri-SOR sweeps (Sec. 2); overwrites the work vectors."""
        _check(load().hz_trisor_apply(self._h, prec, sweeps, omega, _ptr(r), _ptr(z)), "hz_trisor_apply")

    def precond_matvec(self, p, ph, v, prec):
        _check(load().hz_precond_matvec(self._h, prec, _ptr(p), _ptr(ph), _ptr(v)), "hz_precond_matvec")

    def residual(self, b, x, r=None):
        rn, bn = ctypes.c_double(), ctypes.c_double()
        _check(load().hz_residual(self._h, _ptr(b), _ptr(x), _ptr(r), ctypes.byref(rn), ctypes.byref(bn)),
               "hz_residual")
        return rn.value, bn.value

    def autotune(self, fp64=True, trisor=False):
        """Pick the column-kernel variants for this grid from timed trials on the GPU: the fastest,
        unless the measured default is within 2% of it (a stable choice; the dot products'
        rounding, hence the iteration count, follows the variant)."""
        _check(load().hz_op_autotune(self._h, (1 if fp64 else 0) | (2 if trisor else 0)), "hz_op_autotune")
        return self.variants()

    def sor_variants(self):
        """{(prec, kind): id} of the tri-SOR kernels (kind 0 pass, 1 matvec, 2 first pass)."""
        L = load()
        out = {}
        for prec in (HZ_PREC_FP32, HZ_PREC_FP64):
            for kind in range(3):
                v = ctypes.c_int()
                _check(L.hz_op_get_sor_variant(self._h, prec, kind, ctypes.byref(v)), "hz_op_get_sor_variant")
                out[(prec, kind)] = v.value
        return out

    def set_sor_variant(self, prec, kind, id_):
        _check(load().hz_op_set_sor_variant(self._h, prec, kind, id_), "hz_op_set_sor_variant")

    def variants(self):
        v = [ctypes.c_int() for _ in range(4)]
        _check(load().hz_op_get_variants(self._h, *[ctypes.byref(x) for x in v]), "hz_op_get_variants")
        return {"pre32": v[0].value, "mv32": v[1].value, "pre64": v[2].value, "mv64": v[3].value}

    def set_variants(self, pre32=-1, mv32=-1, pre64=-1, mv64=-1):
        _check(load().hz_op_set_variants(self._h, pre32, mv32, pre64, mv64), "hz_op_set_variants")

    def profile(self, on=True):
        _check(load().hz_profile_enable(self._h, 1 if on else 0), "hz_profile_enable")

    def profile_read(self):
        """{kernel name: (launches, ms, algorithmic bytes)} accumulated since profile(True)."""
        L = load()
        out = {}
        for k in range(NUM_KERNELS):
            la, ms, by = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
            _check(L.hz_profile_read(self._h, k, ctypes.byref(la), ctypes.byref(ms), ctypes.byref(by)),
                   "hz_profile_read")
            out[L.hz_kernel_name(k).decode()] = (la.value, ms.value, by.value)
        return out

    def set_band_format(self, fmt):
        """Storage of the horizontal bands for the FP32 BiCGStab kernels: HZ_BANDS_FP32, _BF16 or _FP16."""
        _check(load().hz_op_set_band_format(self._h, int(fmt)), "hz_op_set_band_format")

    def band_format(self):
        v = ctypes.c_int()
        _check(load().hz_op_get_band_format(self._h, ctypes.byref(v)), "hz_op_get_band_format")
        return v.value

    def export(self, what, prec, dst):
        _check(load().hz_op_export(self._h, what, prec, _ptr(dst)), "hz_op_export")


def solve_batched(ops, bs, xs, x0s=None, params=None, raise_on_error=True, strategy=0, **kw):
    """Solve several systems (each its own Operator) in one batched call; returns a list of info dicts.
    strategy: HZ_BATCH_AUTO (0), HZ_BATCH_PERSISTENT (1) or HZ_BATCH_SEQUENTIAL (2)."""
    L = load()
    k = len(ops)
    p = params if params is not None else default_params(**kw)
    arr = ctypes.c_void_p * k
    hs = arr(*[o.handle.value for o in ops])
    bp = arr(*[_ptr(b) for b in bs])
    xp = arr(*[_ptr(x) for x in xs])
    x0p = arr(*[_ptr(x) for x in x0s]) if x0s is not None else None
    infos = (hz_solve_info * k)()
    st = L.hz_solve_batched_ex(k, hs, bp, x0p, xp, ctypes.byref(p), infos, int(strategy))
    out = [i.as_dict() for i in infos]
    if st != HZ_OK and raise_on_error:
        raise HzError(st, f"hz_solve_batched {out}")
    return out if raise_on_error else (st, out)


def batched_debug(timeout_ns=0, leave_block=-1):
    """Test hook: bound of the batched grid-barrier waits and a block that leaves early."""
    _check(load().hz_batched_debug(int(timeout_ns), int(leave_block)), "hz_batched_debug")


def batched_set_vec(vec=0):
    """Columns per thread of the persistent batched kernel: 1 or 4, 0 to choose per batch."""
    _check(load().hz_batched_set_vec(int(vec)), "hz_batched_set_vec")


def dot(x, y, prec=None, stream=None):
    """Deterministic FP64-accumulated dot product of two CUDA tensors."""
    import torch

    if prec is None:
        prec = HZ_PREC_FP32 if x.dtype == torch.float32 else HZ_PREC_FP64
    out = ctypes.c_double()
    _check(load().hz_dot(prec, x.numel(), _ptr(x), _ptr(y), _stream_ptr(stream), ctypes.byref(out)), "hz_dot")
    return out.value


def dot_noalloc(x, y, out, prec=None, stream=None):
    """hz_dot_noalloc: the dot product of two CUDA tensors written to the CUDA
    tensor ``out`` (one float64), using only the library's static scratch (no
    device allocation).  Does not synchronise."""
    import torch

    if prec is None:
        prec = HZ_PREC_FP32 if x.dtype == torch.float32 else HZ_PREC_FP64
    assert out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1
    _check(load().hz_dot_noalloc(prec, x.numel(), _ptr(x), _ptr(y), _stream_ptr(stream), _ptr(out)),
           "hz_dot_noalloc")


def sor_variant_count(prec, kind) -> int:
    return load().hz_sor_variant_count(prec, kind)


def version() -> int:
    return load().hz_version()


# ---- learned preconditioner stage ---------------------------------------------------
class hz_nn_train_params(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int),
        ("batch", ctypes.c_int),
        ("crop", ctypes.c_int),
        ("n_iterates", ctypes.c_int),
        ("iterates", ctypes.c_int * 16),
        ("xstar_tol", ctypes.c_double),
        ("lr", ctypes.c_double),
        ("clip", ctypes.c_double),
        ("seed", ctypes.c_ulonglong),
        ("stream", ctypes.c_ulonglong),
        ("loss", ctypes.c_int),
    ]


def _nn_sigs(L):
    i32, dbl, pv = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "hz_nn_num_params": (i32, []),
        "hz_nn_last_error": (ctypes.c_char_p, []),
        "hz_nn_create": (i32, [pv, P(pv)]),
        "hz_nn_destroy": (i32, [pv]),
        "hz_nn_set_params": (i32, [pv, pv]),
        "hz_nn_get_params": (i32, [pv, pv]),
        "hz_nn_forward": (i32, [pv, i32, i32, i32, i32, i32, pv, pv, pv]),
        "hz_nn_gradient": (i32, [pv, i32, i32, i32, i32, i32, i32, pv, pv, pv, P(dbl)]),
        "hz_nn_train_step": (i32, [pv, i32, i32, i32, i32, i32, i32, pv, pv, dbl, dbl, P(dbl)]),
        "hz_nn_crops": (i32, [i32, i32, i32, pv, pv, i32, i32, i32, pv, pv, pv, pv]),
        "hz_nn_save": (i32, [pv, ctypes.c_char_p]),
        "hz_nn_load": (i32, [pv, ctypes.c_char_p]),
        "hz_op_set_nn": (i32, [pv, pv]),
        "hz_nn_make_pair": (i32, [pv, pv, pv, pv, pv, pv, P(dbl)]),
        "hz_nn_train_defaults": (None, [P(hz_nn_train_params)]),
        "hz_nn_train": (i32, [pv, pv, pv, P(hz_nn_train_params), pv]),
        "hz_nn_gradient_op": (i32, [pv, i32, i32, i32, i32, i32, pv, pv, pv, pv, P(dbl)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _nnlib():
    L = load()
    if not getattr(L, "_nn_ready", False):
        _nn_sigs(L)
        L._nn_ready = True
    return L


def _nn_check(st, where):
    if st != HZ_OK:
        L = _nnlib()
        raise HzError(st, f"{where}: {L.hz_nn_last_error().decode()}")


class Net:
    """The learned preconditioner stage (hz_nn): 4-layer 3-D conv net, BF16 weights and activations."""

    def __init__(self, params=None, stream=None):
        L = _nnlib()
        self._h = ctypes.c_void_p()
        _nn_check(L.hz_nn_create(_stream_ptr(stream), ctypes.byref(self._h)), "hz_nn_create")
        if params is not None:
            self.set_params(params)

    @staticmethod
    def num_params():
        return _nnlib().hz_nn_num_params()

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _nnlib().hz_nn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32) if isinstance(params, np.ndarray) else params
        _nn_check(_nnlib().hz_nn_set_params(self._h, _ptr(p)), "hz_nn_set_params")

    def get_params(self):
        out = np.empty(self.num_params(), dtype=np.float32)
        _nn_check(_nnlib().hz_nn_get_params(self._h, out.ctypes.data), "hz_nn_get_params")
        return out

    def forward(self, x, y, dims, seg_ny=None, periodic=True, zout=None):
        nx, ny, nz = dims
        _nn_check(_nnlib().hz_nn_forward(self._h, nx, ny, nz, seg_ny or ny, int(periodic), _ptr(x), _ptr(y), _ptr(zout)),
                  "hz_nn_forward")

    def gradient(self, x, t, dims, seg_ny=None, periodic=False, border=0):
        nx, ny, nz = dims
        g = np.empty(self.num_params(), dtype=np.float64)
        loss = ctypes.c_double()
        _nn_check(_nnlib().hz_nn_gradient(self._h, nx, ny, nz, seg_ny or ny, int(periodic), border, _ptr(x), _ptr(t),
                                          g.ctypes.data, ctypes.byref(loss)), "hz_nn_gradient")
        return g, loss.value

    def train_step(self, x, t, dims, lr=1e-3, seg_ny=None, periodic=False, border=0, clip=0.0):
        nx, ny, nz = dims
        loss = ctypes.c_double()
        _nn_check(_nnlib().hz_nn_train_step(self._h, nx, ny, nz, seg_ny or ny, int(periodic), border, _ptr(x), _ptr(t),
                                            lr, clip, ctypes.byref(loss)), "hz_nn_train_step")
        return loss.value

    def gradient_op(self, x, t, bands, dims, seg_ny=None, border=5):
        """Gradient and value of the operator-weighted loss on stacked crops (hz_nn_gradient_op)."""
        nx, ny, nz = dims
        g = np.empty(self.num_params(), dtype=np.float64)
        loss = ctypes.c_double()
        _nn_check(_nnlib().hz_nn_gradient_op(self._h, nx, ny, nz, seg_ny or ny, border, _ptr(x), _ptr(t), _ptr(bands),
                                             g.ctypes.data, ctypes.byref(loss)), "hz_nn_gradient_op")
        return g, loss.value

    def train(self, op, b, iterates=None, **kw):
        """hz_nn_train: pairs from the system (op, b) and kw["steps"] Adam steps on crops of them.
        kw: fields of hz_nn_train_params (steps, batch, crop, xstar_tol, lr, clip, seed, stream, loss).
        Returns the losses of the steps."""
        L = _nnlib()
        p = hz_nn_train_params()
        L.hz_nn_train_defaults(ctypes.byref(p))
        if iterates is not None:
            its = list(iterates)
            p.n_iterates = len(its)
            for q, k in enumerate(its):
                p.iterates[q] = int(k)
        for k, v in kw.items():
            if not hasattr(p, k):
                raise KeyError(k)
            setattr(p, k, v)
        out = np.zeros(max(1, p.steps))
        _nn_check(L.hz_nn_train(self._h, op.handle, _ptr(b), ctypes.byref(p), out.ctypes.data), "hz_nn_train")
        return out[: p.steps].tolist()

    def save(self, path):
        _nn_check(_nnlib().hz_nn_save(self._h, str(path).encode()), "hz_nn_save")

    def load(self, path):
        _nn_check(_nnlib().hz_nn_load(self._h, str(path).encode()), "hz_nn_load")


def nn_crops(fa, fb, dims, corners, cx, cy, oa, ob, stream=None):
    """Crops (cx x cy columns, all levels) of two fields at the given (i0, j0) corners, stacked along j."""
    nx, ny, nz = dims
    c = np.ascontiguousarray(np.asarray(corners, dtype=np.int32).reshape(-1))
    _nn_check(_nnlib().hz_nn_crops(nx, ny, nz, _ptr(fa), _ptr(fb), c.size // 2, cx, cy, c.ctypes.data, _ptr(oa),
                                   _ptr(ob), _stream_ptr(stream)), "hz_nn_crops")


def _op_set_nn(self, net):
    _check(_nnlib().hz_op_set_nn(self._h, net.handle if net is not None else None), "hz_op_set_nn")


def _op_make_pair(self, b, xk, xstar, inp, tgt):
    sig = ctypes.c_double()
    _check(_nnlib().hz_nn_make_pair(self._h, _ptr(b), _ptr(xk), _ptr(xstar), _ptr(inp), _ptr(tgt), ctypes.byref(sig)),
           "hz_nn_make_pair")
    return sig.value


Operator.set_nn = _op_set_nn
Operator.make_pair = _op_make_pair
