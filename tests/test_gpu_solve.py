"""End-to-end parity of the GPU solve (through the C ABI) with the CPU oracle.

Bar: the true FP64 relative residual ||b - A x|| / ||b||, recomputed by the
oracle from the GPU's x, is <= tol (1e-8); the solution agrees with the
oracle's FP64 solution (tol 1e-12) to a relative 2-norm difference <= 1e-6.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

SMALL = [(96, 72, 20), (37, 23, 9), (6, 5, 4), (33, 17, 1)]


def _hz():
    import paper_1811_03852_gb300 as hz

    return hz


def _solve(A, b, **kw):
    import torch

    hz = _hz()
    op = hz.Operator(A)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(dev(b), x, **kw)
    return host(x).reshape(b.shape), info, op


@pytest.mark.parametrize("shape", SMALL)
@pytest.mark.parametrize("z_unit", ["radius", "m"])
@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_solve_matches_oracle(shape, z_unit, mode):
    hz = _hz()
    nx, ny, nz = shape
    A, b = gen.make_system(nx, ny, nz, 1, 2, z_unit=z_unit)
    m = hz.HZ_MODE_MIXED_IR if mode == "mixed" else hz.HZ_MODE_FP64
    x, info, _ = _solve(A, b, mode=m, tol=1e-8)
    assert info["status"] == 0
    _, rn = oracle.residual(A, b, x)
    R = rn / np.linalg.norm(b)
    assert R <= 1e-8, R
    # the two residuals differ by rounding: |fl(b - A x) - (b - A x)| <~ n_terms eps |A||x|
    floor = 16 * 2.2e-16 * np.linalg.norm(oracle.matvec(np.abs(A), np.abs(x)) + np.abs(b)) / np.linalg.norm(b)
    assert abs(R - info["true_rel_residual"]) <= 1e-6 * R + floor
    x_ref, ref_info = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-12, eta=1e-13)
    assert ref_info["status"] == 0
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-6


@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_fp64_iteration_count_matches_oracle(z_unit):
    hz = _hz()
    A, b = gen.make_system(96, 72, 20, 1, 2, z_unit=z_unit)
    _, info, _ = _solve(A, b, mode=hz.HZ_MODE_FP64, tol=1e-8, inner_tol=1e-9)
    _, ref = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-8, eta=1e-9)
    # identical algorithm; over hundreds of iterations the rounding-order
    # differences of the reductions move the count by a few percent
    assert info["outer_iters"] == ref["outer"]
    assert abs(info["inner_iters"] - ref["inner"]) <= max(2, 0.12 * ref["inner"]), (info, ref)


def test_graph_and_host_loop_agree_bitwise():
    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 5, 6, z_unit="m")
    xg, ig, _ = _solve(A, b, use_graph=1)
    xe, ie, _ = _solve(A, b, use_graph=0)
    assert ig["inner_iters"] == ie["inner_iters"] and np.array_equal(xg, xe)


def test_repeated_solves_are_deterministic():
    import torch

    hz = _hz()
    A, b = gen.make_system(96, 72, 20, 7, 8, z_unit="m")
    op = hz.Operator(A)
    bd = dev(b)
    outs = []
    for _ in range(3):
        x = torch.empty(b.size, dtype=torch.float64, device="cuda")
        op.solve(bd, x)
        outs.append(host(x))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_host_buffers_and_warm_start_in_place():
    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 9, 10)
    op = hz.Operator(A)  # coefficients from host memory
    x = np.zeros_like(b)
    info = op.solve(b, x)  # b and x in host memory
    assert info["status"] == 0
    _, rn = oracle.residual(A, b, x)
    assert rn / np.linalg.norm(b) <= 1e-8
    # warm start with x0 aliasing x: already converged, no refinement step
    info2 = op.solve(b, x, x0=x)
    assert info2["status"] == 0 and info2["outer_iters"] == 0 and info2["inner_iters"] == 0


def test_zero_rhs_gives_zero():
    import torch

    hz = _hz()
    A = gen.make_operator(8, 6, 5, seed=1)
    op = hz.Operator(A)
    x = torch.full((240,), 7.0, dtype=torch.float64, device="cuda")
    info = op.solve(torch.zeros(240, dtype=torch.float64, device="cuda"), x)
    assert info["status"] == 0 and not torch.any(x)


def test_operator_validation():
    hz = _hz()
    A = gen.make_operator(6, 5, 4, seed=2)
    bad = A.copy()
    bad[3, 0, 4, 0] = -1.0  # N coefficient on the north polar row
    with pytest.raises(hz.HzError) as e:
        hz.Operator(bad)
    assert e.value.status == hz.HZ_ERR_INVALID
    bad = A.copy()
    bad[0, 1, 1, 1] = 0.0  # zero diagonal
    with pytest.raises(hz.HzError):
        hz.Operator(bad)
    bad = A.copy()
    bad[6, 0, 2, 2] = -1.0  # D coefficient through the bottom
    with pytest.raises(hz.HzError):
        hz.Operator(bad)


def test_limits_report_not_converged_with_best_iterate():
    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 11, 12, z_unit="m")
    x, info, _ = _solve(A, b, max_outer=1, max_inner=3, raise_on_error=False)
    assert info["status"] == hz.HZ_ERR_NOT_CONVERGED
    _, rn = oracle.residual(A, b, x)
    assert abs(rn / np.linalg.norm(b) - info["true_rel_residual"]) <= 1e-9 and info["true_rel_residual"] < 1.0


@pytest.mark.parametrize("scale", [1e-36, 1e36])
def test_fp32_range_failure_is_retried_in_fp64(scale):
    # A right-hand side outside the 32-bit range: at 1e-36 the scaled FP32
    # inner right-hand side D^-1 r underflows (the inner solve sees nothing and
    # the refinement step stalls), at 1e36 the FP32 dot products overflow (the
    # inner solve turns non-finite).  The FP64 outer residual is fine in both,
    # and the solver retries once with FP64 inner solves.  A x = b is linear,
    # so the answer is the oracle's solution of the unscaled system times scale.
    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 1, 2)
    x, info, _ = _solve(A, b * scale, raise_on_error=False)
    assert info["status"] == hz.HZ_OK and info["fp64_retries"] == 1, info
    _, rn = oracle.residual(A, b * scale, x)
    assert rn / np.linalg.norm(b * scale) <= 1e-8
    x_ref, _ = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-12, eta=1e-13)
    assert np.linalg.norm(x / scale - x_ref) / np.linalg.norm(x_ref) <= 1e-6
    # in FP64 mode nothing is retried; the plain scale needs no retry either
    _, info64, _ = _solve(A, b * scale, mode=hz.HZ_MODE_FP64)
    assert info64["fp64_retries"] == 0
    _, info1, _ = _solve(A, b)
    assert info1["fp64_retries"] == 0


def test_stall_after_the_fp64_retry_is_not_converged():
    # one inner iteration per refinement step cannot halve R on the hard family:
    # the first stall switches to FP64 inner solves, the next ends the solve
    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 11, 12, z_unit="m")
    x, info, _ = _solve(A, b, max_inner=1, raise_on_error=False)
    assert info["status"] == hz.HZ_ERR_NOT_CONVERGED and info["fp64_retries"] == 1, info
    _, rn = oracle.residual(A, b, x)
    assert abs(rn / np.linalg.norm(b) - info["true_rel_residual"]) <= 1e-9


def test_nonfinite_rhs_reported():
    hz = _hz()
    A, b = gen.make_system(8, 6, 5, 1, 2)
    b[2, 3, 4] = np.nan
    _, info, _ = _solve(A, b, raise_on_error=False)
    assert info["status"] == hz.HZ_ERR_NONFINITE


def test_forced_restarts_still_converge():
    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 13, 14, z_unit="m")
    x, info, _ = _solve(A, b, restart=5)
    assert info["status"] == 0 and info["restarts"] > 0
    _, rn = oracle.residual(A, b, x)
    assert rn / np.linalg.norm(b) <= 1e-8


def test_history_and_fp32_stall_vs_refinement():
    # Sec. 3: a 32-bit Krylov solve alone cannot be trusted below eps_32; the
    # outer FP64 loop reaches 1e-8 where a single FP32 inner solve does not.
    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 15, 16, z_unit="m")
    x1, one, op = _solve(A, b, max_outer=1, inner_tol=1e-10, max_inner=600, record_history=1, raise_on_error=False)
    h = op.history()
    assert len(h) == one["inner_iters"] > 0
    _, rn = oracle.residual(A, b, x1)
    assert rn / np.linalg.norm(b) > 1e-8
    x2, ir, _ = _solve(A, b)
    assert ir["status"] == 0 and ir["outer_iters"] >= 2


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_full_size_640x480x70_true_residual(mode):
    # the 640x480x70 workload at full size: the oracle recomputes the true
    # residual of the GPU solution over every point
    hz = _hz()
    A, b = gen.make_system(640, 480, 70, 11, 12)
    m = hz.HZ_MODE_MIXED_IR if mode == "mixed" else hz.HZ_MODE_FP64
    x, info, _ = _solve(A, b, mode=m)
    assert info["status"] == 0
    _, rn = oracle.residual(A, b, x)
    assert rn / np.linalg.norm(b) <= 1e-8
    # the two residuals agree up to the rounding floor of b - A x (about 1e-15 relative here)
    assert abs(rn / np.linalg.norm(b) - info["true_rel_residual"]) <= 1e-3 * info["true_rel_residual"] + 1e-14


def test_full_size_n1280_true_residual():
    # the N1280-shaped workload (2560x1920x70), launched as the benchmark does
    import torch

    hz = _hz()
    nx, ny, nz = 2560, 1920, 70
    A = gen.make_operator(nx, ny, nz, 21)
    b = gen.make_rhs(nx, ny, nz, 22)
    op = hz.Operator(A)
    bd = dev(b)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(bd, x)
    assert info["status"] == 0
    xh = host(x).reshape(b.shape)
    del x, bd
    _, rn = oracle.residual(A, b, xh)
    R = rn / np.linalg.norm(b)
    assert R <= 1e-8 and abs(R - info["true_rel_residual"]) <= 1e-3 * R
