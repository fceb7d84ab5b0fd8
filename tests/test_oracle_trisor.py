"""Pins for the oracle's tri-SOR preconditioner (Sec. 2: (T + w L) x_n = (1 - w) T x_(n-1) + w (r - U x_(n-1)))."""
import numpy as np
import pytest

import gen
import oracle
from conftest import dense_from_hat


def _split(Ah):
    """Dense T, L, U of Ahat in the red-black column order (colour (i + j) mod 2, red first):
    L = horizontal couplings of black rows to red columns, U = all other horizontal couplings."""
    _, nz, ny, nx = Ah.shape
    M = dense_from_hat(Ah)
    Av = Ah.copy()
    Av[:4] = 0.0
    T = dense_from_hat(Av)
    H = M - T
    colour = np.array([(i + j) % 2 for k in range(nz) for j in range(ny) for i in range(nx)])
    Lmask = (colour[:, None] == 1) & (colour[None, :] == 0)
    L = np.where(Lmask, H, 0.0)
    return T, L, H - L


@pytest.mark.parametrize("shape", [(6, 4, 3), (5, 4, 3), (8, 6, 5)])
@pytest.mark.parametrize("sweeps,omega", [(1, 1.5), (3, 1.5), (2, 1.0)])
def test_trisor_matches_dense_fixed_point(shape, sweeps, omega):
    nx, ny, nz = shape
    Ah = oracle.scale(gen.make_operator(nx, ny, nz, seed=2, z_unit="m"))
    r = gen.normals(3, 0, nx * ny * nz)
    T, L, U = _split(Ah)
    x = np.zeros_like(r)
    for _ in range(sweeps):
        x = np.linalg.solve(T + omega * L, (1 - omega) * T @ x + omega * (r - U @ x))
    z = oracle.apply_trisor(Ah, r.reshape(nz, ny, nx), sweeps, omega).ravel()
    assert np.allclose(z, x, rtol=1e-11, atol=1e-12 * np.abs(x).max())


def test_trisor_without_horizontal_coupling_is_scaled_Tinv():
    nx, ny, nz = 6, 4, 5
    A = gen.make_operator(nx, ny, nz, seed=4)
    A[1:5] = 0.0
    Ah = oracle.scale(A)
    r = gen.normals(5, 0, nx * ny * nz).reshape(nz, ny, nx)
    # one sweep from zero with L = U = 0 gives omega T^-1 r; BiCGStab is invariant to a
    # scalar multiple of its preconditioner, so omega drops out of a T^-1 solve
    assert np.allclose(oracle.apply_trisor(Ah, r, 1, 1.5), 1.5 * oracle.apply_Tinv(Ah, r), rtol=1e-13)


def test_many_sweeps_converge_to_the_solve():
    nx, ny, nz = 8, 6, 4
    Ah = oracle.scale(gen.make_operator(nx, ny, nz, seed=6))
    r = gen.normals(7, 0, nx * ny * nz)
    z = oracle.apply_trisor(Ah, r.reshape(nz, ny, nx), 200, 1.0).ravel()
    assert np.allclose(z, np.linalg.solve(dense_from_hat(Ah), r), rtol=1e-10, atol=1e-12)


def test_bicgstab_with_trisor_solves_and_needs_fewer_iterations():
    nx, ny, nz = 24, 18, 10
    A, b = gen.make_system(nx, ny, nz, 8, 9, z_unit="m")
    Ah = oracle.scale(A)
    bh = b / A[0]
    try:
        oracle.set_precond(1, 3, 1.5)
        x, info = oracle.bicgstab(Ah, bh, eta=1e-12, maxit=2000)
    finally:
        oracle.set_precond(0)
    _, plain = oracle.bicgstab(Ah, bh, eta=1e-12, maxit=2000)
    assert info["status"] == 0 and info["iters"] < plain["iters"]
    assert np.linalg.norm(oracle.matvec_hat(Ah, x) - bh) <= 1e-10 * np.linalg.norm(bh)
