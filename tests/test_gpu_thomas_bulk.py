"""The bulk-copy Thomas variant (inputs staged into shared memory by cp.async.bulk,
forward sweep parked in shared memory) against the register-pipelined one.

Both compute the same recurrences in the same order (Sec. 2's per-column LU
of T, with the fused vector updates), so every output agrees bit for bit,
and so does a whole solve: the same iterates, the same iteration count.
Shapes cover a ragged last tile (columns not a multiple of 256), a single
level, a tile narrower than a warp, and the 640x480x70 workload.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

BULKS = (13, 14, 15, 16, 17)  # the FP32 Thomas variants with park mode 3 (ring of 5, 3, 4 slots; 5 and 8 at one block per SM)
BULK = 13
PLAIN = 10  # the default FP32 Thomas variant


def _hz():
    import paper_1811_03852_gb300 as hz

    return hz


@pytest.mark.parametrize("shape", [(100, 26, 7), (256, 1, 70), (4, 1, 1), (96, 72, 20), (640, 480, 70)])
def test_bulk_variant_is_bitwise_the_plain_one(shape):
    import torch

    hz = _hz()
    nx, ny, nz = shape
    n = nx * ny * nz
    A = gen.make_operator(nx, ny, nz, 3, z_unit="m")
    op = hz.Operator(A)
    L = hz.load()
    p = dev(gen.normals(41, 0, n), torch.float32)
    out = {}
    for var in (PLAIN,) + BULKS:
        assert L.hz_op_set_variants(op.handle, var, -1, -1, -1) == 0
        z = torch.empty(n, dtype=torch.float32, device="cuda")
        ph = torch.empty_like(z)
        v = torch.empty_like(z)
        op.precond_apply(p, z, hz.HZ_PREC_FP32)
        op.precond_matvec(p, ph, v, hz.HZ_PREC_FP32)
        out[var] = (host(z), host(ph), host(v))
    for bulk in BULKS:
        for a, b in zip(out[PLAIN], out[bulk]):
            assert np.array_equal(a, b), bulk
    # and the oracle's T^-1 of the FP32 operator
    Ah = oracle.scale(A).astype(np.float32).astype(np.float64)
    ref = oracle.apply_Tinv(Ah, host(p).astype(np.float64).reshape(nz, ny, nx))
    assert np.max(np.abs(out[BULK][0].reshape(nz, ny, nx) - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("case", [((96, 72, 20), "m"), ((128, 96, 70), "radius")])
def test_bulk_variant_solve_is_bitwise_the_plain_one(case):
    import torch

    hz = _hz()
    shape, z_unit = case
    A, b = gen.make_system(*shape, 5, 6, z_unit=z_unit)
    L = hz.load()
    res = {}
    for var in (PLAIN,) + BULKS:
        op = hz.Operator(A)
        assert L.hz_op_set_variants(op.handle, var, -1, -1, -1) == 0
        x = torch.empty(b.size, dtype=torch.float64, device="cuda")
        info = op.solve(dev(b), x)
        assert info["status"] == 0
        res[var] = (host(x), info["inner_iters"], info["outer_iters"])
        # the host-driven loop (every launch separate) gives the same bits too
        xe = torch.empty_like(x)
        op.solve(dev(b), xe, use_graph=0)
        assert torch.equal(x, xe)
    for bulk in BULKS:
        assert res[PLAIN][1:] == res[bulk][1:]
        assert np.array_equal(res[PLAIN][0], res[bulk][0])
    _, rn = oracle.residual(A, b, res[BULK][0].reshape(b.shape))
    assert rn / np.linalg.norm(b) <= 1e-8


def test_bulk_variant_needs_whole_vectors_of_columns():
    # the copies move rows of 16-byte units: nx * ny must be a multiple of 4
    hz = _hz()
    A = gen.make_operator(37, 23, 9, 3)
    op = hz.Operator(A)
    for bulk in BULKS:
        assert hz.load().hz_op_set_variants(op.handle, bulk, -1, -1, -1) == hz.HZ_ERR_INVALID
