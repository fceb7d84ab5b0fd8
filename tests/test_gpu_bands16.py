"""16-bit storage of the horizontal bands on the GPU (BF16 / FP16, FP32 arithmetic).

The paper's case for 32-bit numbers (Secs. 1 and 3: smaller data moves less)
carried to the four horizontal bands of D^-1 A that the stencil kernels read
twice per inner iteration.  Checks: the stored 16-bit patterns equal the
oracle's rounding bit for bit; the stencil with 16-bit bands equals the
oracle's matvec with the rounded bands; the refinement loop still reaches the
true FP64 residual 1e-8 of the exact A (recomputed by the oracle), with the
solution of the oracle's FP64 solve; formats switch and update cleanly.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import abs_matvec_hat, dev, host

pytestmark = pytest.mark.gpu

FMTS = {"bf16": 1, "fp16": 2}


def _hz():
    import paper_1811_03852_gb300 as hz

    return hz


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
@pytest.mark.parametrize("shape", [(37, 23, 9), (64, 32, 70)])
def test_stored_bands_are_the_oracle_rounding(fmt, shape):
    import torch

    hz = _hz()
    nx, ny, nz = shape
    n = nx * ny * nz
    A = gen.make_operator(nx, ny, nz, 3, z_unit="m")
    op = hz.Operator(A)
    op.set_band_format(FMTS[fmt])
    assert op.band_format() == FMTS[fmt]
    out = torch.empty(4 * n, dtype=torch.int16, device="cuda")
    op.export(2, hz.HZ_PREC_FP32, out)
    got = host(out).view(np.uint16).reshape(4, nz, ny, nx)
    Ah = oracle.scale(A)
    ref = oracle.bits16(oracle.round_hbands(Ah, FMTS[fmt])[:4], FMTS[fmt])
    assert np.array_equal(got, ref)
    # a coefficient update redoes the copies
    A2 = gen.make_operator(nx, ny, nz, 4, z_unit="m")
    op.update(A2)
    op.export(2, hz.HZ_PREC_FP32, out)
    ref2 = oracle.bits16(oracle.round_hbands(oracle.scale(A2), FMTS[fmt])[:4], FMTS[fmt])
    assert np.array_equal(host(out).view(np.uint16).reshape(4, nz, ny, nx), ref2)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
@pytest.mark.parametrize("shape", [(37, 23, 9), (64, 32, 70), (130, 20, 12)])
def test_stencil_with_16bit_bands(fmt, shape):
    # v = p + H16 T^-1 p equals Ahat16 (T^-1 p) with Ahat16 the operator whose
    # horizontal bands are the rounded ones (FP32 tolerance of the other tests)
    import torch

    hz = _hz()
    nx, ny, nz = shape
    n = nx * ny * nz
    A = gen.make_operator(nx, ny, nz, 3, z_unit="m")
    op = hz.Operator(A)
    op.set_band_format(FMTS[fmt])
    Ar = oracle.round_hbands(oracle.scale(A), FMTS[fmt]).astype(np.float32).astype(np.float64)
    p = gen.normals(13, 0, n).reshape(nz, ny, nx).astype(np.float32).astype(np.float64)
    ph = torch.empty(n, dtype=torch.float32, device="cuda")
    v = torch.empty(n, dtype=torch.float32, device="cuda")
    op.precond_matvec(dev(p, torch.float32), ph, v, hz.HZ_PREC_FP32)
    ref_ph = oracle.apply_Tinv(Ar, p)
    ref_v = oracle.matvec_hat(Ar, ref_ph)
    scale = abs_matvec_hat(Ar, ref_ph) + np.abs(p)
    assert np.max(np.abs(host(v).reshape(nz, ny, nx) - ref_v) / scale) <= 1e-5
    # and the full matvec entry point reads the same bands
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    op.matvec(dev(p, torch.float32), y, hz.HZ_PREC_FP32)
    ref_y = oracle.matvec_hat(Ar, p)
    assert np.max(np.abs(host(y).reshape(nz, ny, nx) - ref_y) / abs_matvec_hat(Ar, p)) <= 1e-6


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
@pytest.mark.parametrize("case", [((96, 72, 20), "m"), ((96, 72, 20), "radius"), ((128, 96, 70), "radius")])
def test_refinement_with_16bit_bands_matches_oracle(fmt, case):
    import torch

    hz = _hz()
    shape, z_unit = case
    A, b = gen.make_system(*shape, 1, 2, z_unit=z_unit)
    op = hz.Operator(A)
    op.set_band_format(FMTS[fmt])
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(dev(b), x, max_outer=20)
    xh = host(x).reshape(b.shape)
    _, rn = oracle.residual(A, b, xh)
    assert info["status"] == 0 and rn / np.linalg.norm(b) <= 1e-8, info
    x_ref, _ = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-12, eta=1e-13, max_inner=20000)
    assert np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref) <= 1e-6
    # the oracle's refinement with the same rounded inner operator takes about as many steps
    Ar = oracle.round_hbands(oracle.scale(A), FMTS[fmt]).astype(np.float32)
    _, io = oracle.solve(A, b, mode=oracle.MODE_MIXED, tol=1e-8, inner_bands=Ar, max_outer=20)
    assert io["status"] == 0 and abs(info["outer_iters"] - io["outer"]) <= 1, (info, io)


def test_format_switch_and_paper_solver():
    # back to FP32: the same bits as an operator that never left it (the captured
    # inner loop is rebuilt); the paper's mixed-precision solver reads the format too
    import torch

    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 5, 6, z_unit="m")
    ref_op = hz.Operator(A)
    op = hz.Operator(A)
    x0 = torch.empty(b.size, dtype=torch.float64, device="cuda")
    x1 = torch.empty_like(x0)
    ref_op.solve(dev(b), x0)
    op.set_band_format(hz.HZ_BANDS_BF16)
    # 8 significant bits slow the refinement on this hard system: more than the default 10 steps
    i16 = op.solve(dev(b), x1, max_outer=30)
    assert i16["status"] == 0, i16
    op.set_band_format(hz.HZ_BANDS_FP32)
    i32 = op.solve(dev(b), x1)
    assert torch.equal(x0, x1) and i32["status"] == 0
    op.set_band_format(hz.HZ_BANDS_FP16)
    mp = op.solve(dev(b), x1, mode=hz.HZ_MODE_PAPER_MP, tol=1e-4)
    assert mp["status"] == 0
    with pytest.raises(hz.HzError):
        op.set_band_format(7)


@pytest.mark.parametrize("fmt", ["bf16", "fp16"])
def test_full_size_640x480x70(fmt):
    import torch

    hz = _hz()
    A, b = gen.make_system(640, 480, 70, 11, 12)
    op = hz.Operator(A)
    op.set_band_format(FMTS[fmt])
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(dev(b), x, max_outer=20)
    _, rn = oracle.residual(A, b, host(x).reshape(b.shape))
    assert info["status"] == 0 and rn / np.linalg.norm(b) <= 1e-8, info
