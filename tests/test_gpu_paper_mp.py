"""The paper's own mixed-precision solver (HZ_MODE_PAPER_MP) on the GPU, and its Sec. 4 observations.

HZ_MODE_PAPER_DP is the 64-bit solver it is compared with: the same single
solve and halting test in FP64.

Sec. 3: the solver works in 32-bit while the pressure field x stays 64-bit;
there is no refinement.  Sec. 4 compares it with the 64-bit solver on the
same systems: after one iteration the two residuals agree to about seven
significant figures; both reach the operational halting criterion R_c = 1e-3
in the same number of iterations (Table 1: 8.4 and 8.4; 29.3 and 29.3 at
1e-4); the global sums, first 32-bit, were reverted to 64-bit because
near-zero scalars made the solver fail.  Here: the same comparisons on the
synthetic hard system (metres unit) and on 640x480x70, against the oracle's
paper-MP and FP64 BiCGStab (the oracle counts are the same algorithm in
another summation order, so they are matched within a tolerance).
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _hz():
    import paper_1811_03852_gb300 as hz

    return hz


def _solve(op, b, **kw):
    import torch

    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(dev(b), x, raise_on_error=False, **kw)
    return host(x).reshape(b.shape), info


def test_paper_mp_matches_the_oracle():
    hz = _hz()
    A, b = gen.make_system(96, 72, 20, 1, 2, z_unit="m")
    op = hz.Operator(A)
    for rc in (1e-3, 1e-4):
        x, info = _solve(op, b, mode=hz.HZ_MODE_PAPER_MP, tol=rc)
        assert info["status"] == hz.HZ_OK and info["outer_iters"] == 1 and info["fp64_retries"] == 0, info
        assert info["scaled_rel_residual"] <= rc
        xo, io = oracle.solve(A, b, mode=oracle.MODE_PAPER_MP, tol=rc, eta=rc)
        assert io["outer"] == 1
        assert abs(info["inner_iters"] - io["inner"]) <= max(2, 0.15 * io["inner"]), (info, io)
        # the library's report is the FP64 R of the x it returned
        _, rn = oracle.residual(A, b, x)
        assert info["true_rel_residual"] == pytest.approx(rn / np.linalg.norm(b), rel=1e-6)
        # same algorithm, same halting test: about the same point of the iteration
        # (the FP64 R moves by tens of percent from one iteration to the next here)
        assert io["R"] / 3 <= info["true_rel_residual"] <= 3 * io["R"], (info, io)


@pytest.mark.parametrize("pre", ["tri", "trisor"])
def test_sec4_mixed_and_double_precision_agree_to_rc_1e3(pre):
    # one iteration: seven significant figures; R_c = 1e-3: identical counts
    hz = _hz()
    pc = hz.HZ_PRE_TRISOR if pre == "trisor" else hz.HZ_PRE_TRI
    A, b = gen.make_system(96, 72, 20, 1, 2, z_unit="m")
    op = hz.Operator(A)
    hist = {}
    counts = {}
    for name, mode in (("mp", hz.HZ_MODE_PAPER_MP), ("dp", hz.HZ_MODE_PAPER_DP)):
        _, info = _solve(op, b, mode=mode, precond=pc, tol=1e-3, record_history=1)
        assert info["status"] == hz.HZ_OK
        counts[name] = info["inner_iters"]
        hist[name] = op.history()
    assert abs(hist["mp"][0] - hist["dp"][0]) <= 1e-6 * hist["dp"][0], (hist["mp"][:3], hist["dp"][:3])
    assert counts["mp"] == counts["dp"], counts
    # at the halting iteration (22 on this hard system, against 8.4 in Table 1)
    # the two residuals still agree to within a few percent (measured 2%; the
    # paper's milder systems agree to four significant figures)
    k = counts["mp"] - 1
    assert abs(hist["mp"][k] - hist["dp"][k]) <= 5e-2 * hist["dp"][k]


def test_table1_counts_at_rc_1e4_and_32bit_global_sums():
    # R_c = 1e-4: counts within a few iterations (Table 1: identical means);
    # with every dot product summed in FP32 (the original global sums) the solver
    # still converges on this system: the overflow the paper met with near-zero
    # scalars does not occur here (reported, not forced)
    hz = _hz()
    A, b = gen.make_system(96, 72, 20, 1, 2, z_unit="m")
    op = hz.Operator(A)
    _, mp = _solve(op, b, mode=hz.HZ_MODE_PAPER_MP, tol=1e-4)
    _, dp = _solve(op, b, mode=hz.HZ_MODE_PAPER_DP, tol=1e-4)
    _, mp32 = _solve(op, b, mode=hz.HZ_MODE_PAPER_MP, tol=1e-4, dot_fp32=1)
    for i in (mp, dp, mp32):
        assert i["status"] == hz.HZ_OK, i
    assert abs(mp["inner_iters"] - dp["inner_iters"]) <= max(2, 0.15 * dp["inner_iters"]), (mp, dp)
    assert abs(mp32["inner_iters"] - mp["inner_iters"]) <= max(2, 0.15 * mp["inner_iters"]), (mp32, mp)


def test_fp32_sums_change_the_rounding_not_the_solve():
    # the FP32 global sums give different scalars (different bits) but the same
    # converged answer through the refinement loop
    import torch

    hz = _hz()
    A, b = gen.make_system(37, 23, 9, 1, 2, z_unit="m")
    op = hz.Operator(A)
    x1, i1 = _solve(op, b)
    x2, i2 = _solve(op, b, dot_fp32=1)
    assert i1["status"] == i2["status"] == hz.HZ_OK
    for x in (x1, x2):
        _, rn = oracle.residual(A, b, x)
        assert rn / np.linalg.norm(b) <= 1e-8
    _, ih1 = _solve(op, b, mode=hz.HZ_MODE_PAPER_MP, tol=1e-5, record_history=1)
    h1 = op.history()
    _, ih2 = _solve(op, b, mode=hz.HZ_MODE_PAPER_MP, tol=1e-5, record_history=1, dot_fp32=1)
    h2 = op.history()
    assert not np.array_equal(h1, h2)  # the switch reaches the reductions
    assert abs(h1[0] - h2[0]) <= 1e-5 * h1[0]
    del torch


def test_paper_mp_640x480x70_and_its_limit():
    # the Earth-radius system of 640x480x70: identical counts at 1e-3 and 1e-4
    # (the oracle's own MP and FP64 solvers agree there: 4/4 and 6/6); and the
    # paper's point that 32 bits alone cannot reach 1e-8: the same solver asked
    # for 1e-8 stops on its recursive residual with the FP64 R far above it,
    # where the refinement loop reaches it
    hz = _hz()
    A, b = gen.make_system(640, 480, 70, 11, 12)
    op = hz.Operator(A)
    for rc in (1e-3, 1e-4):
        _, mp = _solve(op, b, mode=hz.HZ_MODE_PAPER_MP, tol=rc)
        _, dp = _solve(op, b, mode=hz.HZ_MODE_PAPER_DP, tol=rc)
        assert mp["status"] == dp["status"] == hz.HZ_OK
        assert mp["inner_iters"] == dp["inner_iters"], (rc, mp, dp)
        assert mp["true_rel_residual"] == pytest.approx(dp["true_rel_residual"], rel=1e-2)
    _, mp8 = _solve(op, b, mode=hz.HZ_MODE_PAPER_MP, tol=1e-8, max_inner=300)
    _, ir = _solve(op, b, tol=1e-8)
    assert mp8["true_rel_residual"] > 1e-7, mp8
    assert ir["status"] == hz.HZ_OK and ir["true_rel_residual"] <= 1e-8


def test_paper_mp_rejections_and_host_buffers():
    hz = _hz()
    A, b = gen.make_system(16, 12, 6, 1, 2)
    op = hz.Operator(A)
    x = np.empty_like(b)
    with pytest.raises(hz.HzError):
        op.solve(b, x, mode=hz.HZ_MODE_PAPER_MP, krylov=hz.HZ_KRYLOV_FGMRES)
    with pytest.raises(hz.HzError):
        op.solve(b, x, mode=hz.HZ_MODE_FP64, dot_fp32=1)
    with pytest.raises(hz.HzError):
        op.solve(b, x, mode=hz.HZ_MODE_PAPER_DP, dot_fp32=1)
    info = op.solve(b, x, mode=hz.HZ_MODE_PAPER_MP, tol=1e-6)  # host b and x
    _, rn = oracle.residual(A, b, x)
    assert info["true_rel_residual"] == pytest.approx(rn / np.linalg.norm(b), rel=1e-6)
