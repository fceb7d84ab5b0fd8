"""Parity of the tri-SOR preconditioner (Sec. 2) on the GPU with the CPU oracle.

Preconditioner alone (hz_trisor_apply, gather -> colour passes -> scatter):
FP64 within 1e-12 and FP32 within 1e-5 of max|z| against the oracle's
red-black sweeps (FP32: oracle on the FP32-rounded operator and input).
Solver: true FP64 relative residual <= 1e-8 recomputed by the oracle, the
solution within 1e-6 of the oracle's FP64 solution, and the FP64 inner
iteration count within 12% of the oracle's tri-SOR BiCGStab.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

# nx even (red-black needs it); several tiles, ragged tails, nx = 2, one level
SHAPES = [(96, 72, 20), (38, 23, 9), (6, 5, 4), (2, 3, 5), (130, 65, 11), (34, 17, 1)]


def _hz():
    import paper_1811_03852_gb300 as hz

    return hz


def _solve(A, b, **kw):
    import torch

    hz = _hz()
    op = hz.Operator(A)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    kw.setdefault("precond", hz.HZ_PRE_TRISOR)
    info = op.solve(dev(b), x, **kw)
    return host(x).reshape(b.shape), info, op


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("sweeps,omega", [(3, 1.5), (1, 1.0), (2, 0.7)])
def test_trisor_apply_matches_oracle(shape, prec, sweeps, omega):
    import torch

    hz = _hz()
    nx, ny, nz = shape
    A = gen.make_operator(nx, ny, nz, seed=4, z_unit="m")
    op = hz.Operator(A)
    Ah = oracle.scale(A)
    r = gen.normals(6, 0, nx * ny * nz).reshape(nz, ny, nx)
    if prec == "fp64":
        z = torch.empty(r.size, dtype=torch.float64, device="cuda")
        op.trisor_apply(dev(r), z, hz.HZ_PREC_FP64, sweeps, omega)
        zo = oracle.apply_trisor(Ah, r, sweeps, omega)
        tol = 1e-12
    else:
        z = torch.empty(r.size, dtype=torch.float32, device="cuda")
        r32 = r.astype(np.float32)
        op.trisor_apply(dev(r32), z, hz.HZ_PREC_FP32, sweeps, omega)
        zo = oracle.apply_trisor(Ah.astype(np.float32).astype(np.float64), r32.astype(np.float64), sweeps, omega)
        tol = 1e-5
    zg = host(z).astype(np.float64).reshape(r.shape)
    assert np.max(np.abs(zg - zo)) <= tol * np.max(np.abs(zo))


def test_trisor_one_sweep_omega_one_is_block_jacobi_gauss_seidel():
    # one sweep with omega = 1 from zero: red columns get T^-1 r exactly, black
    # columns T^-1 (r - H z_red) -- checked against T^-1 applied by the oracle
    import torch

    hz = _hz()
    nx, ny, nz = 38, 23, 9
    A = gen.make_operator(nx, ny, nz, seed=8, z_unit="m")
    op = hz.Operator(A)
    Ah = oracle.scale(A)
    r = gen.normals(9, 0, nx * ny * nz).reshape(nz, ny, nx)
    z = torch.empty(r.size, dtype=torch.float64, device="cuda")
    op.trisor_apply(dev(r), z, hz.HZ_PREC_FP64, 1, 1.0)
    zg = host(z).reshape(r.shape)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    red = ((i + j) % 2 == 0)[None].repeat(nz, 0)
    zt = oracle.apply_Tinv(Ah, r)
    assert np.max(np.abs(zg[red] - zt[red])) <= 1e-13 * np.max(np.abs(zt))
    zr = np.where(red, zg, 0.0)
    # on black rows, (Ahat - I) z_red is H z_red: U and D stay inside a column, which is zero there
    h = oracle.matvec_hat(Ah, zr) - zr
    zb = oracle.apply_Tinv(Ah, r - h)
    assert np.max(np.abs(zg[~red] - zb[~red])) <= 1e-12 * np.max(np.abs(zb))


@pytest.mark.parametrize("shape", [(96, 72, 20), (38, 23, 9), (6, 5, 4)])
@pytest.mark.parametrize("z_unit", ["radius", "m"])
@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_solve_trisor_matches_oracle(shape, z_unit, mode):
    hz = _hz()
    nx, ny, nz = shape
    A, b = gen.make_system(nx, ny, nz, 1, 2, z_unit=z_unit)
    m = hz.HZ_MODE_MIXED_IR if mode == "mixed" else hz.HZ_MODE_FP64
    x, info, _ = _solve(A, b, mode=m, tol=1e-8)
    assert info["status"] == 0
    _, rn = oracle.residual(A, b, x)
    R = rn / np.linalg.norm(b)
    assert R <= 1e-8, R
    floor = 16 * 2.2e-16 * np.linalg.norm(oracle.matvec(np.abs(A), np.abs(x)) + np.abs(b)) / np.linalg.norm(b)
    assert abs(R - info["true_rel_residual"]) <= 1e-6 * R + floor
    x_ref, ref_info = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-12, eta=1e-13)
    assert ref_info["status"] == 0
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-6


@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_fp64_trisor_iteration_count_matches_oracle(z_unit):
    hz = _hz()
    A, b = gen.make_system(96, 72, 20, 1, 2, z_unit=z_unit)
    _, info, _ = _solve(A, b, mode=hz.HZ_MODE_FP64, tol=1e-8, inner_tol=1e-9)
    oracle.set_precond(1, 3, 1.5)
    try:
        _, ref = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-8, eta=1e-9)
    finally:
        oracle.set_precond(0)
    assert info["outer_iters"] == ref["outer"]
    assert abs(info["inner_iters"] - ref["inner"]) <= max(2, 0.12 * ref["inner"]), (info, ref)


def test_trisor_needs_fewer_iterations_than_tinv():
    # Sec. 2: the horizontal coupling that T^-1 ignores is what tri-SOR adds
    hz = _hz()
    A, b = gen.make_system(96, 72, 20, 3, 4, z_unit="m")
    _, it, _ = _solve(A, b, precond=hz.HZ_PRE_TRI)
    _, isor, _ = _solve(A, b)
    assert it["status"] == 0 and isor["status"] == 0
    assert isor["inner_iters"] < it["inner_iters"]


def test_trisor_graph_host_loop_and_profile_agree_bitwise():
    import torch

    hz = _hz()
    A, b = gen.make_system(38, 23, 9, 5, 6, z_unit="m")
    xg, ig, _ = _solve(A, b, use_graph=1)
    xe, ie, _ = _solve(A, b, use_graph=0)
    assert ig["inner_iters"] == ie["inner_iters"] and np.array_equal(xg, xe)
    op = hz.Operator(A)
    op.profile(True)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    ip = op.solve(dev(b), x, precond=hz.HZ_PRE_TRISOR)
    prof = op.profile_read()
    op.profile(False)
    assert ip["inner_iters"] == ig["inner_iters"] and np.array_equal(host(x).reshape(b.shape), xg)
    for k in ("k_sor_first", "k_sor_pass", "k_mv_rb", "k_rb_copy", "k_upd"):
        assert prof[k][0] > 0, (k, prof)
    assert prof["k_pre_p"][0] == 0
    assert ip["kernel_launches"] == sum(v[0] for v in prof.values())


def test_trisor_repeated_solves_are_deterministic():
    import torch

    hz = _hz()
    A, b = gen.make_system(96, 72, 20, 7, 8, z_unit="m")
    op = hz.Operator(A)
    bd = dev(b)
    outs = []
    for _ in range(3):
        x = torch.empty(b.size, dtype=torch.float64, device="cuda")
        op.solve(bd, x, precond=hz.HZ_PRE_TRISOR)
        outs.append(host(x))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_trisor_after_update_uses_new_coefficients():
    import torch

    hz = _hz()
    A1, b = gen.make_system(38, 23, 9, 11, 12, z_unit="m")
    A2 = gen.make_operator(38, 23, 9, 13, z_unit="m")
    op = hz.Operator(A1)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    op.solve(dev(b), x, precond=hz.HZ_PRE_TRISOR)
    op.update(A2)
    info = op.solve(dev(b), x, precond=hz.HZ_PRE_TRISOR)
    _, rn = oracle.residual(A2, b, host(x).reshape(b.shape))
    assert info["status"] == 0 and rn / np.linalg.norm(b) <= 1e-8


def test_trisor_forced_restarts_warm_start_and_sweep_counts():
    hz = _hz()
    A, b = gen.make_system(38, 23, 9, 13, 14, z_unit="m")
    x, info, op = _solve(A, b, restart=3)
    assert info["status"] == 0 and info["restarts"] > 0
    _, rn = oracle.residual(A, b, x)
    assert rn / np.linalg.norm(b) <= 1e-8
    xw = x.copy()
    info2 = op.solve(b, xw, x0=xw, precond=hz.HZ_PRE_TRISOR)
    assert info2["status"] == 0 and info2["outer_iters"] == 0
    for sweeps, omega in [(1, 1.0), (2, 1.2), (5, 1.5)]:
        xs, inf, _ = _solve(A, b, sor_sweeps=sweeps, sor_omega=omega)
        assert inf["status"] == 0
        _, rn = oracle.residual(A, b, xs)
        assert rn / np.linalg.norm(b) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_pass_variant_gives_identical_columns(prec):
    # the variants change only launch shape and load batching, not the arithmetic of a column
    import torch

    hz = _hz()
    nx, ny, nz = 136, 65, 11  # nx/2 = 68: every vector width fits; ragged ny
    A = gen.make_operator(nx, ny, nz, seed=4, z_unit="m")
    op = hz.Operator(A)
    p = hz.HZ_PREC_FP64 if prec == "fp64" else hz.HZ_PREC_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    r = dev(gen.normals(6, 0, nx * ny * nz), dt)
    outs = []
    for vid in range(hz.sor_variant_count(p, 0)):
        op.set_sor_variant(p, 0, vid)
        z = torch.empty(r.numel(), dtype=dt, device="cuda")
        op.trisor_apply(r, z, p, 3, 1.5)
        outs.append(host(z))
    assert len(outs) >= 3 and all(np.array_equal(outs[0], o) for o in outs[1:])
    zo = oracle.apply_trisor(oracle.scale(A) if prec == "fp64" else oracle.scale(A).astype(np.float32).astype(np.float64),
                             host(r).astype(np.float64).reshape(nz, ny, nx), 3, 1.5)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert np.max(np.abs(outs[0].astype(np.float64).reshape(zo.shape) - zo)) <= tol * np.max(np.abs(zo))


def test_variants_wider_than_the_row_are_rejected():
    hz = _hz()
    A = gen.make_operator(130, 9, 5, seed=4)  # nx/2 = 65: only one column per thread fits
    op = hz.Operator(A)
    for p in (hz.HZ_PREC_FP32, hz.HZ_PREC_FP64):
        ok = []
        for vid in range(hz.sor_variant_count(p, 0)):
            try:
                op.set_sor_variant(p, 0, vid)
                ok.append(vid)
            except hz.HzError as e:
                assert e.status == hz.HZ_ERR_INVALID
        assert 0 in ok and len(ok) < hz.sor_variant_count(p, 0)


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_every_matvec_and_first_pass_variant_solves(mode):
    hz = _hz()
    A, b = gen.make_system(96, 72, 20, 1, 2, z_unit="m")
    m = hz.HZ_MODE_MIXED_IR if mode == "mixed" else hz.HZ_MODE_FP64
    p = hz.HZ_PREC_FP32 if mode == "mixed" else hz.HZ_PREC_FP64
    x_ref, _ = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-12, eta=1e-13)
    import torch

    op = hz.Operator(A)
    for kind in (1, 2):
        for vid in range(hz.sor_variant_count(p, kind)):
            op.set_sor_variant(p, kind, vid)
            x = torch.empty(b.size, dtype=torch.float64, device="cuda")
            info = op.solve(dev(b), x, mode=m, precond=hz.HZ_PRE_TRISOR)
            xh = host(x).reshape(b.shape)
            _, rn = oracle.residual(A, b, xh)
            assert info["status"] == 0 and rn / np.linalg.norm(b) <= 1e-8, (kind, vid)
            assert np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref) <= 1e-6
        op.set_sor_variant(p, kind, 0)


def test_autotune_picks_valid_sor_variants_and_solves():
    import torch

    hz = _hz()
    A, b = gen.make_system(96, 72, 20, 3, 4, z_unit="m")
    op = hz.Operator(A)
    op.autotune(fp64=True, trisor=True)
    v = op.sor_variants()
    for (prec, kind), vid in v.items():
        assert 0 <= vid < hz.sor_variant_count(prec, kind)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(dev(b), x, precond=hz.HZ_PRE_TRISOR)
    _, rn = oracle.residual(A, b, host(x).reshape(b.shape))
    assert info["status"] == 0 and rn / np.linalg.norm(b) <= 1e-8
    with pytest.raises(hz.HzError):
        op.set_sor_variant(hz.HZ_PREC_FP32, 0, hz.sor_variant_count(hz.HZ_PREC_FP32, 0))


def test_trisor_rejections():
    import torch

    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 1, 2)  # nx odd
    op = hz.Operator(A)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    with pytest.raises(hz.HzError) as e:
        op.solve(dev(b), x, precond=hz.HZ_PRE_TRISOR)
    assert e.value.status == hz.HZ_ERR_UNSUPPORTED
    with pytest.raises(hz.HzError) as e:
        op.trisor_apply(dev(b), x, hz.HZ_PREC_FP64)
    assert e.value.status == hz.HZ_ERR_UNSUPPORTED
    A, b = gen.make_system(38, 23, 9, 1, 2)
    op = hz.Operator(A)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    with pytest.raises(hz.HzError) as e:
        op.solve(dev(b), x, precond=hz.HZ_PRE_TRISOR, krylov=hz.HZ_KRYLOV_FGMRES)
    assert e.value.status == hz.HZ_ERR_UNSUPPORTED
    for kw in ({"sor_sweeps": 0}, {"sor_sweeps": 65}, {"sor_omega": 0.0}, {"sor_omega": 2.0}):
        with pytest.raises(hz.HzError) as e:
            op.solve(dev(b), x, precond=hz.HZ_PRE_TRISOR, **kw)
        assert e.value.status == hz.HZ_ERR_INVALID


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_trisor_full_size_640x480x70_true_residual(mode):
    hz = _hz()
    A, b = gen.make_system(640, 480, 70, 11, 12)
    m = hz.HZ_MODE_MIXED_IR if mode == "mixed" else hz.HZ_MODE_FP64
    x, info, _ = _solve(A, b, mode=m)
    assert info["status"] == 0
    _, rn = oracle.residual(A, b, x)
    assert rn / np.linalg.norm(b) <= 1e-8
    assert abs(rn / np.linalg.norm(b) - info["true_rel_residual"]) <= 1e-3 * info["true_rel_residual"] + 1e-14


def test_trisor_full_size_n1280_true_residual():
    import torch

    hz = _hz()
    nx, ny, nz = 2560, 1920, 70
    A = gen.make_operator(nx, ny, nz, 21)
    b = gen.make_rhs(nx, ny, nz, 22)
    op = hz.Operator(A)
    bd = dev(b)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(bd, x, precond=hz.HZ_PRE_TRISOR)
    assert info["status"] == 0
    xh = host(x).reshape(b.shape)
    del x, bd
    _, rn = oracle.residual(A, b, xh)
    R = rn / np.linalg.norm(b)
    assert R <= 1e-8 and abs(R - info["true_rel_residual"]) <= 1e-3 * R
