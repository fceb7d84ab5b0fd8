"""Pins for the CPU oracle: each check compares it with something other than itself.

Dense LAPACK solves (numpy.linalg.solve), banded LAPACK solves
(scipy.linalg.solve_banded), closed forms and brute force on tiny grids.
"""
import numpy as np
import pytest
import scipy.linalg

import gen
import oracle
from conftest import dense_from_hat, dense_operator

TINY = [(4, 4, 3), (6, 5, 4), (5, 3, 1), (3, 2, 7)]


@pytest.mark.parametrize("shape", TINY)
@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_matvec_matches_dense_assembly(shape, z_unit):
    nx, ny, nz = shape
    A = gen.make_operator(nx, ny, nz, seed=3, z_unit=z_unit)
    x = gen.normals(7, 0, nx * ny * nz).reshape(nz, ny, nx)
    M = dense_operator(A)
    y_ref = M @ x.ravel()
    y = oracle.matvec(A, x).ravel()
    scale = np.abs(M) @ np.abs(x.ravel())
    assert np.max(np.abs(y - y_ref) / scale) < 1e-15 * 8


@pytest.mark.parametrize("shape", TINY)
def test_matvec_row_sums_closed_form(shape):
    # diagonal = -(sum of off-diagonals) + c  =>  A * 1 = c * 1 exactly up to rounding
    nx, ny, nz = shape
    A = gen.make_operator(nx, ny, nz, seed=5)
    c = A.sum(axis=0).ravel()
    assert np.allclose(c, c[0], rtol=1e-12)
    y = oracle.matvec(A, np.ones((nz, ny, nx)))
    assert np.allclose(y.ravel(), c[0], rtol=1e-9 * np.abs(A).max() / c[0])


def test_matvec_periodic_wrap_brute_force():
    # single unit impulse at i = 0: the west neighbour of i = 0 is i = nx-1
    nx, ny, nz = 5, 3, 2
    A = gen.make_operator(nx, ny, nz, seed=9)
    x = np.zeros((nz, ny, nx))
    x[1, 1, 0] = 1.0
    y = oracle.matvec(A, x)
    assert y[1, 1, nx - 1] == A[1, 1, 1, nx - 1]  # E band of the point east-adjacent across the seam
    assert y[1, 1, 1] == A[2, 1, 1, 1]  # W band of i = 1
    assert y[1, 1, 0] == A[0, 1, 1, 0]
    assert y[0, 1, 0] == A[5, 0, 1, 0]  # U band of the level below
    assert y[1, 2, 0] == A[4, 1, 2, 0]  # S band of the row above
    assert np.count_nonzero(y) == 7 - 1  # the impulse sits on the top level: no U neighbour above


def test_scale_is_diagonal_scaling():
    nx, ny, nz = 4, 4, 3
    A = gen.make_operator(nx, ny, nz, seed=4)
    Ah = oracle.scale(A)
    M = dense_operator(A)
    Mh = np.diag(1.0 / np.diag(M)) @ M
    assert np.allclose(np.diag(Mh), 1.0)
    assert np.allclose(dense_from_hat(Ah), Mh, rtol=1e-15, atol=1e-17)
    x = gen.normals(1, 1, nx * ny * nz).reshape(nz, ny, nx)
    assert np.allclose(oracle.matvec_hat(Ah, x).ravel(), Mh @ x.ravel(), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("m", [1, 2, 3, 20, 70])
def test_tridiag_vs_lapack(m):
    rng = np.random.default_rng(m)
    lo = rng.uniform(-0.4, 0, m)
    up = rng.uniform(-0.4, 0, m)
    lo[0] = 0.0
    up[-1] = 0.0
    di = 1.0 + rng.uniform(0, 0.2, m)
    r = rng.standard_normal(m)
    x = oracle.tridiag_solve(lo, di, up, r)
    T = np.diag(di) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
    assert np.allclose(x, np.linalg.solve(T, r), rtol=1e-13, atol=1e-14)
    ab = np.zeros((3, m))
    ab[0, 1:] = up[:-1]
    ab[1] = di
    ab[2, :-1] = lo[1:]
    assert np.allclose(x, scipy.linalg.solve_banded((1, 1), ab, r), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("shape", [(4, 4, 3), (6, 5, 4), (3, 2, 9)])
@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_apply_Tinv_vs_dense_block_solve(shape, z_unit):
    nx, ny, nz = shape
    A = gen.make_operator(nx, ny, nz, seed=6, z_unit=z_unit)
    Ah = oracle.scale(A)
    r = gen.normals(2, 0, nx * ny * nz).reshape(nz, ny, nx)
    z = oracle.apply_Tinv(Ah, r)
    # T = vertical part of Ahat: keep only the U and D bands
    Ahv = Ah.copy()
    Ahv[:4] = 0.0
    T = dense_from_hat(Ahv)
    assert np.allclose(z.ravel(), np.linalg.solve(T, r.ravel()), rtol=1e-12, atol=1e-13)


def test_Tinv_is_identity_for_one_level():
    nx, ny, nz = 6, 5, 1
    Ah = oracle.scale(gen.make_operator(nx, ny, nz, seed=2))
    r = gen.normals(3, 0, nx * ny).reshape(1, ny, nx)
    assert np.array_equal(oracle.apply_Tinv(Ah, r), r)


@pytest.mark.parametrize("shape", [(4, 4, 3), (6, 5, 4)])
@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_bicgstab_vs_dense_lu(shape, z_unit):
    nx, ny, nz = shape
    A, b = gen.make_system(nx, ny, nz, 8, 9, z_unit=z_unit)
    Ah = oracle.scale(A)
    bh = b / A[0]
    x, info = oracle.bicgstab(Ah, bh, eta=1e-14, maxit=500)
    assert info["status"] == 0
    Mh = dense_from_hat(Ah)
    x_lu = np.linalg.solve(Mh, bh.ravel())
    kappa = np.linalg.cond(Mh)
    assert np.linalg.norm(x.ravel() - x_lu) / np.linalg.norm(x_lu) <= max(kappa, 10) * 1e-13


def test_bicgstab_one_iteration_without_horizontal_coupling():
    # E=W=N=S=0 => Ahat = T => right-preconditioned BiCGStab is exact after one half step
    nx, ny, nz = 5, 4, 6
    A, b = gen.make_system(nx, ny, nz, 12, 13)
    A[1:5] = 0.0
    Ah = oracle.scale(A)
    bh = b / A[0]
    x, info = oracle.bicgstab(Ah, bh, eta=1e-12, maxit=50)
    assert info["iters"] == 1 and info["status"] == 0
    Ahv = Ah.copy()
    assert np.allclose(x.ravel(), np.linalg.solve(dense_from_hat(Ahv), bh.ravel()), rtol=1e-12)


def test_manufactured_solution():
    nx, ny, nz = 6, 5, 4
    A = gen.make_operator(nx, ny, nz, seed=14, z_unit="m")
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    xs = (np.cos(2 * np.pi * i / nx) * np.sin(np.pi * (j + 0.5) / ny) * (1 + k / nz)).transpose(2, 1, 0).copy()
    b = (dense_operator(A) @ xs.ravel()).reshape(nz, ny, nx)
    for mode in (oracle.MODE_FP64, oracle.MODE_MIXED):
        x, info = oracle.solve(A, b, mode=mode, tol=1e-12, eta=1e-4 if mode else 1e-13)
        assert info["status"] == 0 and info["R"] <= 1e-12
        kappa = np.linalg.cond(dense_operator(A))
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-12


@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_mixed_ir_outer_residual_monotone_and_exact(z_unit):
    nx, ny, nz = 8, 6, 5
    A, b = gen.make_system(nx, ny, nz, 21, 22, z_unit=z_unit)
    x, info, hist = oracle.solve(A, b, mode=oracle.MODE_MIXED, tol=1e-10, eta=1e-4, history=True)
    assert info["status"] == 0 and info["R"] <= 1e-10
    assert np.all(np.diff(hist) < 0), hist
    x_lu = np.linalg.solve(dense_operator(A), b.ravel())
    kappa = np.linalg.cond(dense_operator(A))
    assert np.linalg.norm(x.ravel() - x_lu) / np.linalg.norm(x_lu) <= kappa * 1e-10
    # true residual recomputed independently
    assert np.linalg.norm(b.ravel() - dense_operator(A) @ x.ravel()) / np.linalg.norm(b) <= 1e-10


def test_fp32_emulation_is_float_and_stalls():
    # Sec. 4 behaviour on a synthetic system: single and double agree after one
    # iteration to about 7 digits (not to 12), and single precision alone
    # cannot reach a residual far below eps_32, while refinement can.
    nx, ny, nz = 12, 8, 6
    A, b = gen.make_system(nx, ny, nz, 31, 32, z_unit="m")
    Ah = oracle.scale(A)
    bh = b / A[0]
    _, i64, h64 = oracle.bicgstab(Ah, bh, eta=1e-30, maxit=1, history=True)
    _, i32, h32 = oracle.bicgstab(Ah, bh, eta=1e-30, maxit=1, fp32=True, history=True)
    rel = abs(h32[0] - h64[0]) / h64[0]
    assert 1e-12 < rel < 1e-5, rel
    x32, deep32 = oracle.bicgstab(Ah, bh, eta=1e-11, maxit=400, fp32=True)
    # the recursive residual may run below eps_32, the true one cannot
    true32 = np.linalg.norm(bh - oracle.matvec_hat(Ah, x32.astype(np.float64))) / np.linalg.norm(bh)
    assert true32 > 1e-9, true32
    x, info = oracle.solve(A, b, mode=oracle.MODE_MIXED, tol=1e-11, eta=1e-4)
    assert info["status"] == 0


def test_restart_period_is_honoured():
    # a restart every 5 iterations must be counted and must not change the answer
    nx, ny, nz = 8, 6, 5
    A, b = gen.make_system(nx, ny, nz, 41, 42, z_unit="m")
    Ah = oracle.scale(A)
    bh = b / A[0]
    x1, i1 = oracle.bicgstab(Ah, bh, eta=1e-12, maxit=2000, restart=5)
    x2, i2 = oracle.bicgstab(Ah, bh, eta=1e-12, maxit=2000, restart=150)
    assert i1["restarts"] >= (i1["iters"] - 1) // 5 and i1["status"] == 0 and i2["status"] == 0
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) < 1e-8


def test_zero_rhs_gives_zero():
    A = gen.make_operator(4, 3, 2, seed=1)
    x, info = oracle.solve(A, np.zeros((2, 3, 4)), mode=oracle.MODE_MIXED)
    assert info["status"] == 0 and not np.any(x)


def _exact_dot(a, b):
    """The exact value of sum_i a_i b_i (every double is a rational number)."""
    from fractions import Fraction

    return sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)), Fraction(0))


@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000])
def test_dot_within_the_recursive_summation_bound(n):
    # Sec. 4's global sums in FP64: a left-to-right sum of n rounded products
    # lies within gamma_n sum|a_i b_i| of the exact value, gamma_n = n u / (1 - n u)
    # (Higham, Accuracy and Stability, Sec. 3.1); n = 0 is the empty sum
    a = gen.normals(61, 0, n)
    b = gen.normals(62, 0, n)
    exact = _exact_dot(a, b)
    got = oracle.dot(a, b)
    u = 2.0**-53
    gamma = (n + 1) * u / (1 - (n + 1) * u)
    bound = gamma * float(np.sum(np.abs(a * b)))
    assert abs(got - float(exact)) <= bound
    if n == 0:
        assert got == 0.0
    if n == 1:
        assert got == a[0] * b[0]  # one rounded product, nothing to add


def test_dot_adversarial_cancellation_and_order():
    # exactly representable partial sums: the result is exact whatever the bound
    a = np.array([3.0, -1.5, 0.25, 2.0**-20])
    b = np.array([2.0, 4.0, -8.0, 2.0**10])
    assert oracle.dot(a, b) == float(_exact_dot(a, b)) == -2.0 + 2.0**-10
    # catastrophic cancellation: summed left to right, 1e16 + 1 rounds (to even) back
    # to 1e16 and the small term is lost, which the error bound allows; with the large
    # terms first they cancel exactly and the small one survives
    b = np.ones(3)
    assert oracle.dot(np.array([1e16, 1.0, -1e16]), b) == 0.0
    assert oracle.dot(np.array([1e16, -1e16, 1.0]), b) == 1.0
    assert float(_exact_dot(np.array([1e16, 1.0, -1e16]), b)) == 1.0
    # a dropped last term or a squared operand would fail these
    a = np.array([1.0, 2.0, 3.0])
    b = np.array([5.0, 7.0, 11.0])
    assert oracle.dot(a, b) == 52.0
    assert oracle.dot(b, a) == 52.0


def test_openmp_build_gives_the_same_bits():
    # the OpenMP build of the oracle (used only to time it on all host cores)
    # shares out independent loops and sums over fixed chunks: any thread count
    # computes the same values as the serial build
    nx, ny, nz = 96, 72, 20  # 138,240 points: the sums span three chunks
    A, b = gen.make_system(nx, ny, nz, 1, 2, z_unit="m")
    Ah = oracle.scale(A)
    try:
        ref = [oracle.residual(A, b, b)[1], oracle.apply_Tinv(Ah, b), oracle.matvec_hat(Ah, b),
               oracle.solve(A, b, mode=oracle.MODE_MIXED, max_inner=60, max_outer=2)[0],
               oracle.apply_trisor(Ah, b, 3, 1.5)]
        for threads in (3, 8):
            assert oracle.use_openmp(True, threads) == threads
            got = [oracle.residual(A, b, b)[1], oracle.apply_Tinv(Ah, b), oracle.matvec_hat(Ah, b),
                   oracle.solve(A, b, mode=oracle.MODE_MIXED, max_inner=60, max_outer=2)[0],
                   oracle.apply_trisor(Ah, b, 3, 1.5)]
            for r, g in zip(ref, got):
                assert np.array_equal(np.asarray(r), np.asarray(g))
    finally:
        oracle.use_openmp(False)


@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_paper_mp_bicgstab_shares_the_fp32_recursion(z_unit):
    # Sec. 3's mixed-precision solver keeps x in FP64 and everything else in
    # FP32.  BiCGStab never reads x between restarts, so without a restart its
    # recursive residuals are the FP32 solver's, bit for bit, and the two
    # iterates differ only by the rounding of x's own updates
    nx, ny, nz = 16, 12, 6
    A, b = gen.make_system(nx, ny, nz, 3, 4, z_unit=z_unit)
    Ah = oracle.scale(A)
    bh = b / A[0]
    x32, i32, h32 = oracle.bicgstab(Ah, bh, eta=1e-5, maxit=200, restart=10**6, fp32=True, history=True)
    x64, i64, h64 = oracle.bicgstab(Ah, bh, eta=1e-5, maxit=200, restart=10**6, fp32=True, x64=True, history=True)
    assert x64.dtype == np.float64 and x32.dtype == np.float32
    assert i32["restarts"] == i64["restarts"] == 0
    assert i32["iters"] == i64["iters"] and np.array_equal(h32, h64)
    assert np.linalg.norm(x64 - x32) <= 1e-5 * np.linalg.norm(x64)


@pytest.mark.parametrize("case", [((4, 4, 3), "radius"), ((6, 5, 4), "radius"), ((4, 4, 3), "m")])
def test_paper_mp_solve_vs_dense_lu(case):
    # one FP32 solve to R_c = 1e-5 with x in FP64 and no refinement (mode 2):
    # on systems whose recursion stays smooth, the residual of the scaled system
    # (Sec. 2 scales by D^-1 outside the solver) recomputed densely in FP64 meets
    # the tolerance up to FP32 rounding, and x is the dense LU solution within
    # the conditioning of that residual
    shape, z_unit = case
    nx, ny, nz = shape
    A, b = gen.make_system(nx, ny, nz, 5, 6, z_unit=z_unit)
    M = dense_operator(A)
    xs = np.linalg.solve(M, b.ravel())
    x, info, hist = oracle.solve(A, b, mode=oracle.MODE_PAPER_MP, tol=1e-5, eta=1e-5, history=True)
    assert info["outer"] == 1 and len(hist) == 2  # one solve, no refinement
    r = b.ravel() - M @ x.ravel()
    assert info["R"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b), rel=1e-9)
    d = A[0].ravel()
    Ms = M / d[:, None]
    rs = np.linalg.norm(r / d) / np.linalg.norm(b.ravel() / d)
    assert rs <= 2e-5
    assert np.linalg.norm(x.ravel() - xs) <= np.linalg.cond(Ms) * 2e-5 * np.linalg.norm(xs)


def test_paper_mp_first_iterations_match_fp64():
    # Sec. 4: after one iteration the mixed-precision and 64-bit solvers agree to
    # about seven significant figures (the precision of a 32-bit number), and
    # they stay close for the first few
    nx, ny, nz = 16, 12, 6
    A, b = gen.make_system(nx, ny, nz, 3, 4, z_unit="m")
    Ah = oracle.scale(A)
    bh = b / A[0]
    _, _, hmp = oracle.bicgstab(Ah, bh, eta=1e-12, maxit=5, fp32=True, x64=True, history=True)
    _, _, h64 = oracle.bicgstab(Ah, bh, eta=1e-12, maxit=5, history=True)
    rel = np.abs(hmp - h64) / h64
    assert rel[0] <= 1e-6 and np.all(rel <= 1e-4), rel
