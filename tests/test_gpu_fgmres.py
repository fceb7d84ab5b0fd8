"""Flexible GMRES(m) inner solver (GPU): the result must meet the same bar as BiCGStab.

The solution is unique, so it is compared with the oracle's FP64 solution
(relative 2-norm <= 1e-6) and its true FP64 residual recomputed by the oracle
(<= 1e-8); the iteration path is not compared.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _solve(A, b, **kw):
    import torch

    import paper_1811_03852_gb300 as hz

    op = hz.Operator(A)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(dev(b), x, **kw)
    return host(x).reshape(b.shape), info


@pytest.mark.parametrize("shape", [(96, 72, 20), (37, 23, 9), (6, 5, 4)])
@pytest.mark.parametrize("z_unit", ["radius", "m"])
@pytest.mark.parametrize("m", [30, 5])
def test_fgmres_matches_oracle(shape, z_unit, m):
    import paper_1811_03852_gb300 as hz

    nx, ny, nz = shape
    A, b = gen.make_system(nx, ny, nz, 1, 2, z_unit=z_unit)
    x, info = _solve(A, b, krylov=hz.HZ_KRYLOV_FGMRES, fgmres_m=m)
    assert info["status"] == 0, info
    _, rn = oracle.residual(A, b, x)
    assert rn / np.linalg.norm(b) <= 1e-8
    x_ref, _ = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-12, eta=1e-13)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-6
    if z_unit == "m" and m == 5 and nx > 6:
        assert info["restarts"] > 0


@pytest.mark.parametrize("k", [3, 10])
def test_fgmres_minimal_residual_property(k):
    # k BiCGStab iterations apply the (fixed) preconditioner 2k times, so their
    # iterate lies in the Krylov space that 2k FGMRES steps minimise over: the
    # FGMRES residual may not be larger (up to FP32 rounding)
    import paper_1811_03852_gb300 as hz

    A, b = gen.make_system(96, 72, 20, 3, 4, z_unit="m")
    _, ig = _solve(A, b, krylov=hz.HZ_KRYLOV_FGMRES, fgmres_m=64, max_outer=1, max_inner=2 * k, inner_tol=1e-12,
                   raise_on_error=False)
    _, ib = _solve(A, b, max_outer=1, max_inner=k, inner_tol=1e-12, raise_on_error=False)
    assert ig["inner_iters"] == 2 * k and ib["inner_iters"] == k
    assert ig["scaled_rel_residual"] <= 1.01 * ib["scaled_rel_residual"], (ig, ib)


def test_fgmres_rejects_fp64_mode_and_bad_m():
    import paper_1811_03852_gb300 as hz

    A, b = gen.make_system(8, 6, 5, 1, 2)
    _, info = _solve(A, b, krylov=hz.HZ_KRYLOV_FGMRES, mode=hz.HZ_MODE_FP64, raise_on_error=False)
    assert info["status"] == hz.HZ_ERR_UNSUPPORTED
    _, info = _solve(A, b, krylov=hz.HZ_KRYLOV_FGMRES, fgmres_m=0, raise_on_error=False)
    assert info["status"] == hz.HZ_ERR_UNSUPPORTED
