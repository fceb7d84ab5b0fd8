"""Pins for the oracle's 16-bit storage of the horizontal bands (the smaller-data
argument of Secs. 1 and 3 carried to 16 bits): the two roundings against the
formats' definitions, and solves with the rounded operator against dense LU."""
import numpy as np
import pytest

import gen
import oracle
from conftest import dense_from_hat, dense_operator


def test_bf16_rounding_follows_the_format():
    # 8 significant bits, FP32 exponent range, ties to even
    exact = np.array([1.0, -0.5, 3.0, 2.0**-100, 1.0 + 2.0**-7, 255.0 * 2.0**-20])
    assert np.array_equal(oracle.round_bf16(exact), exact)
    one = 1.0
    assert oracle.round_bf16(np.array([one + 2.0**-8]))[0] == 1.0  # tie -> even (1.0)
    assert oracle.round_bf16(np.array([one + 3 * 2.0**-8]))[0] == 1.0 + 2.0**-6  # tie -> even (1 + 2^-6)
    assert oracle.round_bf16(np.array([one + 2.0**-8 + 2.0**-20]))[0] == 1.0 + 2.0**-7  # above the tie
    x = gen.normals(71, 0, 20000) * np.exp(gen.normals(72, 0, 20000) * 20)
    r = oracle.round_bf16(x)
    assert np.all(np.abs(r - x) <= 2.0**-8 * np.abs(x) * (1 + 1e-6))  # unit roundoff 2^-8
    o = np.argsort(x)
    assert np.all(np.diff(r[o]) >= 0)  # rounding is monotone
    # the bit patterns are the top halves of the FP32 patterns
    b = oracle.bits16(r, 1)
    assert np.array_equal((b.astype(np.uint32) << 16).view(np.float32).astype(np.float64), r)


def test_fp16_rounding_follows_the_format():
    # 11 significant bits, ties to even, subnormal spacing 2^-24 below 2^-14
    exact = np.array([1.0, -0.5, 2.0**-14, 2.0**-24, 65504.0, 1.0 + 2.0**-10])
    assert np.array_equal(oracle.round_fp16(exact), exact)
    assert oracle.round_fp16(np.array([1.0 + 2.0**-11]))[0] == 1.0
    assert oracle.round_fp16(np.array([1.0 + 3 * 2.0**-11]))[0] == 1.0 + 2.0**-9
    assert oracle.round_fp16(np.array([2.0**-26]))[0] == 0.0
    assert oracle.round_fp16(np.array([3 * 2.0**-25]))[0] == 2.0**-23  # tie between 2^-24 and 2^-23 -> even
    x = gen.normals(73, 0, 20000) * 10.0 ** (gen.normals(74, 0, 20000))
    x = x[np.abs(x) >= 2.0**-14]
    r = oracle.round_fp16(x)
    assert np.all(np.abs(r - x) <= 2.0**-11 * np.abs(x) * (1 + 1e-6))
    assert np.array_equal(oracle.bits16(r, 2).view(np.float16).astype(np.float64), r)


@pytest.mark.parametrize("fmt", [1, 2])
def test_rounded_bands_touch_only_the_horizontal_part(fmt):
    A = gen.make_operator(8, 6, 5, 3, z_unit="m")
    Ah = oracle.scale(A)
    Ar = oracle.round_hbands(Ah, fmt)
    assert np.array_equal(Ar[4:], Ah[4:])  # U, D unchanged
    assert not np.array_equal(Ar[:4], Ah[:4])
    rel = np.abs(Ar[:4] - Ah[:4]) / np.maximum(np.abs(Ah[:4]), 1e-300)
    assert rel[np.abs(Ah[:4]) > 2.0**-14].max() <= (2.0**-8 if fmt == 1 else 2.0**-11) * (1 + 1e-6)


@pytest.mark.parametrize("fmt", [1, 2])
@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_solves_with_rounded_bands(fmt, z_unit):
    nx, ny, nz = 6, 5, 4
    A, b = gen.make_system(nx, ny, nz, 5, 6, z_unit=z_unit)
    Ah = oracle.scale(A)
    Ar = oracle.round_hbands(Ah, fmt)
    bh = b / A[0]
    # the FP64 BiCGStab on the rounded operator solves that operator (dense LU of I + rounded bands)
    y, info = oracle.bicgstab(Ar, bh, eta=1e-12, maxit=500)
    y_ref = np.linalg.solve(dense_from_hat(Ar), bh.ravel())
    assert info["status"] == 0
    assert np.linalg.norm(y.ravel() - y_ref) <= 1e-9 * np.linalg.norm(y_ref)
    # refinement with FP32 inner solves on the rounded operator reaches the true
    # FP64 residual of the exact A: the outer loop sees the unrounded matrix
    x, ir, hist = oracle.solve(A, b, mode=oracle.MODE_MIXED, tol=1e-10, inner_bands=Ar.astype(np.float32),
                               history=True)
    assert ir["status"] == 0 and ir["R"] <= 1e-10
    assert np.all(np.diff(hist) < 0)
    x_ref = np.linalg.solve(dense_operator(A), b.ravel())
    assert np.linalg.norm(x.ravel() - x_ref) <= 1e-7 * np.linalg.norm(x_ref)
