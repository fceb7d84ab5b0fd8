"""Element-by-element parity of the CUDA building blocks (through the C ABI) with the CPU oracle.

Tolerances: FP64 matvec 1e-13 and FP32 matvec 1e-6 relative to |Ahat||x|
elementwise; Thomas FP64 1e-12 and FP32 1e-5 relative to max|z|; FP64
residual 1e-13 relative to |A||x| + |b|.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import abs_matvec_hat, dev, host

pytestmark = pytest.mark.gpu

# several 128-column tiles plus ragged tails (n not a multiple of 4, nx not a multiple of 32)
SHAPES = [(96, 72, 20), (37, 23, 9), (4, 4, 3), (130, 65, 11), (5, 3, 1), (1, 6, 5), (64, 32, 70)]


def _op(nx, ny, nz, seed=3, z_unit="radius"):
    import paper_1811_03852_gb300 as hz

    A = gen.make_operator(nx, ny, nz, seed=seed, z_unit=z_unit)
    return hz, A, hz.Operator(A)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_setup_scaling_and_factors(shape, z_unit):
    import torch

    nx, ny, nz = shape
    hz, A, op = _op(nx, ny, nz, z_unit=z_unit)
    n = nx * ny * nz
    Ah = oracle.scale(A)
    out64 = torch.empty(6 * n, dtype=torch.float64, device="cuda")
    op.export(0, hz.HZ_PREC_FP64, out64)
    g64 = host(out64).reshape(Ah.shape)
    assert np.allclose(g64, Ah, rtol=5e-16, atol=0)
    out32 = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    op.export(0, hz.HZ_PREC_FP32, out32)
    assert np.allclose(host(out32).reshape(Ah.shape), Ah.astype(np.float32), rtol=1.2e-7, atol=0)
    # factors reproduce the oracle's T^-1 when applied by hand in FP64
    th = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    op.export(1, hz.HZ_PREC_FP64, th)
    m, l, cp = host(th).reshape(3, nz, ny, nx)
    r = gen.normals(5, 0, n).reshape(nz, ny, nx)
    y = np.zeros_like(r)
    for k in range(nz):
        y[k] = m[k] * r[k] - (l[k] * y[k - 1] if k else 0.0)
    z = np.zeros_like(r)
    for k in range(nz - 1, -1, -1):
        z[k] = y[k] - (cp[k] * z[k + 1] if k + 1 < nz else 0.0)
    zo = oracle.apply_Tinv(Ah, r)
    assert np.max(np.abs(z - zo)) <= 1e-12 * np.max(np.abs(zo))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_matvec_parity(shape, prec):
    import torch

    nx, ny, nz = shape
    hz, A, op = _op(nx, ny, nz, z_unit="m")
    n = nx * ny * nz
    Ah = oracle.scale(A)
    x = gen.normals(11, 0, n).reshape(nz, ny, nx)
    if prec == "fp64":
        y = torch.empty(n, dtype=torch.float64, device="cuda")
        op.matvec(dev(x), y, hz.HZ_PREC_FP64)
        ref, scale, tol = oracle.matvec_hat(Ah, x), abs_matvec_hat(Ah, x), 1e-13
    else:
        x32, Ah32 = x.astype(np.float32), Ah.astype(np.float32).astype(np.float64)
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        op.matvec(dev(x32), y, hz.HZ_PREC_FP32)
        xd = x32.astype(np.float64)
        ref, scale, tol = oracle.matvec_hat(Ah32, xd), abs_matvec_hat(Ah32, xd), 1e-6
    err = np.abs(host(y).reshape(nz, ny, nx) - ref) / scale
    assert err.max() <= tol, err.max()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_thomas_parity(shape, prec, z_unit):
    import torch

    nx, ny, nz = shape
    hz, A, op = _op(nx, ny, nz, z_unit=z_unit)
    n = nx * ny * nz
    Ah = oracle.scale(A)
    r = gen.normals(12, 0, n).reshape(nz, ny, nx)
    if prec == "fp64":
        z = torch.empty(n, dtype=torch.float64, device="cuda")
        op.precond_apply(dev(r), z, hz.HZ_PREC_FP64)
        ref, tol = oracle.apply_Tinv(Ah, r), 1e-12
    else:
        r32 = r.astype(np.float32)
        z = torch.empty(n, dtype=torch.float32, device="cuda")
        op.precond_apply(dev(r32), z, hz.HZ_PREC_FP32)
        ref, tol = oracle.apply_Tinv(Ah.astype(np.float32).astype(np.float64), r32.astype(np.float64)), 1e-5
    err = np.max(np.abs(host(z).reshape(nz, ny, nx) - ref)) / np.max(np.abs(ref))
    assert err <= tol, err


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_precond_matvec_is_ahat_tinv(shape, prec):
    # v = p + H T^-1 p must equal Ahat (T^-1 p)
    import torch

    nx, ny, nz = shape
    hz, A, op = _op(nx, ny, nz, z_unit="m")
    n = nx * ny * nz
    Ah = oracle.scale(A)
    p = gen.normals(13, 0, n).reshape(nz, ny, nx)
    dt, P, tol = (torch.float64, hz.HZ_PREC_FP64, 1e-12) if prec == "fp64" else (torch.float32, hz.HZ_PREC_FP32, 1e-5)
    if prec == "fp32":
        p = p.astype(np.float32).astype(np.float64)
        Ah = Ah.astype(np.float32).astype(np.float64)
    ph = torch.empty(n, dtype=dt, device="cuda")
    v = torch.empty(n, dtype=dt, device="cuda")
    op.precond_matvec(dev(p, dt), ph, v, P)
    ref_ph = oracle.apply_Tinv(Ah, p)
    ref_v = oracle.matvec_hat(Ah, ref_ph)
    scale = abs_matvec_hat(Ah, ref_ph) + np.abs(p)
    assert np.max(np.abs(host(v).reshape(nz, ny, nx) - ref_v) / scale) <= tol


@pytest.mark.parametrize("shape", SHAPES)
def test_true_residual_parity(shape):
    import torch

    nx, ny, nz = shape
    hz, A, op = _op(nx, ny, nz, z_unit="m")
    n = nx * ny * nz
    b = gen.make_rhs(nx, ny, nz, 4)
    x = gen.normals(14, 0, n).reshape(nz, ny, nx)
    r = torch.empty(n, dtype=torch.float64, device="cuda")
    rn, bn = op.residual(dev(b), dev(x), r)
    ref, rn_ref = oracle.residual(A, b, x)
    scale = oracle.matvec(np.abs(A), np.abs(x)) + np.abs(b)
    assert np.max(np.abs(host(r).reshape(nz, ny, nx) - ref) / scale) <= 1e-13
    assert abs(rn - rn_ref) <= 1e-12 * rn_ref
    assert abs(bn - np.linalg.norm(b)) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("n", [1, 7, 1000, 138240, 1 << 22])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dot_parity_and_determinism(n, prec):
    import torch

    import paper_1811_03852_gb300 as hz

    x = gen.normals(21, 0, n)
    y = gen.normals(22, 0, n)
    dt = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        x, y = x.astype(np.float32).astype(np.float64), y.astype(np.float32).astype(np.float64)
    xd, yd = dev(x, dt), dev(y, dt)
    vals = [hz.dot(xd, yd) for _ in range(10)]
    assert len(set(vals)) == 1, "reduction is not deterministic"
    ref = oracle.dot(x, y)
    assert abs(vals[0] - ref) <= 1e-13 * np.dot(np.abs(x), np.abs(y))


@pytest.mark.parametrize("shape", [(96, 72, 20), (64, 32, 70), (38, 5, 7), (37, 23, 9)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_column_variant_matches_oracle(shape, prec):
    # each launch-shape variant (columns per thread, levels per batch) the
    # autotuner may pick must give the oracle's T^-1 and Ahat T^-1
    import torch

    nx, ny, nz = shape
    hz, A, op = _op(nx, ny, nz, z_unit="m")
    n = nx * ny * nz
    Ah = oracle.scale(A)
    P = hz.HZ_PREC_FP64 if prec == "fp64" else hz.HZ_PREC_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-12 if prec == "fp64" else 1e-5
    p = gen.normals(31, 0, n).reshape(nz, ny, nx)
    if prec == "fp32":
        p = p.astype(np.float32).astype(np.float64)
        Ah = Ah.astype(np.float32).astype(np.float64)
    ref_ph = oracle.apply_Tinv(Ah, p)
    ref_v = oracle.matvec_hat(Ah, ref_ph)
    scale = abs_matvec_hat(Ah, ref_ph) + np.abs(p)
    L = hz.load()
    pi = 1 if prec == "fp64" else 0
    tried = 0
    for var in range(32):  # ids past the table are refused
        for kind in (0, 1):
            args = [-1, -1, -1, -1]
            args[2 * pi + kind] = var
            if L.hz_op_set_variants(op.handle, *args) != 0:
                continue
            tried += 1
            ph = torch.empty(n, dtype=dt, device="cuda")
            v = torch.empty(n, dtype=dt, device="cuda")
            op.precond_matvec(dev(p, dt), ph, v, P)
            eph = np.max(np.abs(host(ph).reshape(nz, ny, nx) - ref_ph)) / np.max(np.abs(ref_ph))
            ev = np.max(np.abs(host(v).reshape(nz, ny, nx) - ref_v) / scale)
            assert eph <= tol and ev <= tol, (var, kind, eph, ev)
    assert tried >= 2


# Thomas variants (kind 0) that park the forward sweep in the output vector
# under L2 priorities (some with a cap on resident blocks) and stencil variants
# (kind 1) that stream under L2 priorities, each paired with the plain variant
# of the same shape (columns per thread, levels per batch)
L2_PAIRS = {"fp32": [(0, 3, 9), (0, 3, 10), (0, 3, 12), (0, 1, 11), (1, 1, 4), (1, 2, 5), (1, 3, 6)],
            "fp64": [(0, 2, 3), (0, 2, 4), (0, 0, 5), (1, 1, 3), (1, 0, 4)]}


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape", [(96, 72, 20), (640, 48, 70), (38, 6, 9)])
def test_l2_priority_variants_match_plain_bitwise(shape, prec):
    # cache priorities and grid caps change where data lives, not the
    # arithmetic: T^-1 p and Ahat T^-1 p agree bit for bit with the plain variant
    import torch

    nx, ny, nz = shape
    hz, A, op = _op(nx, ny, nz, z_unit="m")
    n = nx * ny * nz
    P = hz.HZ_PREC_FP64 if prec == "fp64" else hz.HZ_PREC_FP32
    dt = torch.float64 if prec == "fp64" else torch.float32
    pi = 1 if prec == "fp64" else 0
    p = dev(gen.normals(41, 0, n), dt)
    L = hz.load()

    def run(kind, var):
        args = [-1, -1, -1, -1]
        args[2 * pi + kind] = var
        if L.hz_op_set_variants(op.handle, *args) != 0:
            return None  # the shape's vector width does not divide nx
        ph = torch.empty(n, dtype=dt, device="cuda")
        v = torch.empty(n, dtype=dt, device="cuda")
        op.precond_matvec(p, ph, v, P)
        return host(ph), host(v)

    tried = 0
    for kind, plain, hinted in L2_PAIRS[prec]:
        a = run(kind, plain)
        b = run(kind, hinted)
        assert (a is None) == (b is None), (kind, plain, hinted)
        if a is None:
            continue
        tried += 1
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (kind, plain, hinted)
    assert tried >= 2


def test_autotune_picks_valid_variants_and_solves():
    import torch

    hz, A, op = _op(96, 72, 20, z_unit="m")
    v = op.autotune(fp64=True)
    assert all(x >= 0 for x in v.values())
    b = gen.make_rhs(96, 72, 20, 3)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(dev(b), x)
    _, rn = oracle.residual(A, b, host(x).reshape(b.shape))
    assert info["status"] == 0 and rn / np.linalg.norm(b) <= 1e-8


def test_every_thomas_variant_solves():
    # the solver's own Thomas kernels (k_pre_p, k_pre_s) in every FP32 variant,
    # including those that park the forward sweep in shared memory
    import torch

    import paper_1811_03852_gb300 as hz

    A, b = gen.make_system(96, 72, 20, 5, 6, z_unit="m")
    op = hz.Operator(A)
    L = hz.load()
    x_ref, _ = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-12, eta=1e-13)
    tried = 0
    for var in range(32):  # ids past the table are refused
        if L.hz_op_set_variants(op.handle, var, -1, -1, -1) != 0:
            continue
        tried += 1
        x = torch.empty(b.size, dtype=torch.float64, device="cuda")
        info = op.solve(dev(b), x)
        xh = host(x).reshape(b.shape)
        _, rn = oracle.residual(A, b, xh)
        assert info["status"] == 0 and rn / np.linalg.norm(b) <= 1e-8, var
        assert np.linalg.norm(xh - x_ref) / np.linalg.norm(x_ref) <= 1e-6, var
    assert tried >= 8


def test_every_stencil_variant_solves():
    # the solver's own stencil kernels (k_mv, with their dot products) in every
    # FP32 and FP64 variant, in the mixed and the FP64 solver
    import torch

    import paper_1811_03852_gb300 as hz

    A, b = gen.make_system(96, 72, 20, 7, 8, z_unit="m")
    op = hz.Operator(A)
    L = hz.load()
    tried = 0
    for pi, mode in ((0, hz.HZ_MODE_MIXED_IR), (1, hz.HZ_MODE_FP64)):
        for var in range(32):  # ids past the table are refused
            args = [-1, -1, -1, -1]
            args[2 * pi + 1] = var
            if L.hz_op_set_variants(op.handle, *args) != 0:
                continue
            tried += 1
            x = torch.empty(b.size, dtype=torch.float64, device="cuda")
            info = op.solve(dev(b), x, mode=mode)
            _, rn = oracle.residual(A, b, host(x).reshape(b.shape))
            assert info["status"] == 0 and rn / np.linalg.norm(b) <= 1e-8, (pi, var)
    assert tried >= 10
