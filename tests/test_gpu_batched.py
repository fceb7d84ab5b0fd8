"""Batched solves: the persistent strategy (many uneven systems, or many
right-hand sides of one operator: the whole solve, refinement loop included,
in one cooperative launch, replayable from a CUDA graph) and the sequential
one (hz_solve per system).

Each system of a batch must reach the true FP64 residual 1e-8 (recomputed by
the oracle) and agree with its own single-system solve to 1e-6 (relative 2-norm).
The bounded grid-barrier wait must turn a block that leaves into HZ_ERR_TIMEOUT.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _systems(specs, z_unit="m"):
    out = []
    for (nx, ny, nz, sc, sr) in specs:
        A = gen.make_operator(nx, ny, nz, sc, z_unit=z_unit)
        b = gen.make_rhs(nx, ny, nz, sr)
        out.append((A, b))
    return out


def _batched(systems, **kw):
    import torch

    import paper_1811_03852_gb300 as hz

    ops = [hz.Operator(A) for A, _ in systems]
    bs = [dev(b.reshape(-1)) for _, b in systems]
    xs = [torch.empty(b.size, dtype=torch.float64, device="cuda") for _, b in systems]
    infos = hz.solve_batched(ops, bs, xs, **kw)
    return [host(x).reshape(b.shape) for x, (_, b) in zip(xs, systems)], infos, ops


@pytest.mark.parametrize("z_unit", ["radius", "m"])
def test_batched_uneven_matches_single_solves(z_unit):
    import torch

    specs = [(96, 72, 20, 100 + 2 * i, 101 + 2 * i) if i % 3 == 0 else
             (64, 48, 20, 100 + 2 * i, 101 + 2 * i) if i % 3 == 1 else
             (32, 24, 20, 100 + 2 * i, 101 + 2 * i) for i in range(7)]
    systems = _systems(specs, z_unit)
    xs, infos, ops = _batched(systems)
    for (A, b), x, info, op in zip(systems, xs, infos, ops):
        assert info["status"] == 0, info
        _, rn = oracle.residual(A, b, x)
        assert rn / np.linalg.norm(b) <= 1e-8
        xd = torch.empty(b.size, dtype=torch.float64, device="cuda")
        single = op.solve(dev(b), xd)
        xsgl = host(xd).reshape(b.shape)
        assert np.linalg.norm(x - xsgl) / np.linalg.norm(xsgl) <= 1e-6
        assert single["status"] == 0


def test_batched_scalar_path_and_warm_start():
    # nx not a multiple of 4 -> one column per thread; x0 given for one system
    import torch

    import paper_1811_03852_gb300 as hz

    systems = _systems([(37, 23, 9, 5, 6), (96, 72, 20, 7, 8), (6, 5, 4, 9, 10)])
    ops = [hz.Operator(A) for A, _ in systems]
    bs = [dev(b.reshape(-1)) for _, b in systems]
    xs = [torch.empty(b.size, dtype=torch.float64, device="cuda") for _, b in systems]
    x0s = [None, torch.zeros(systems[1][1].size, dtype=torch.float64, device="cuda"), None]
    infos = hz.solve_batched(ops, bs, xs, x0s=x0s)
    for (A, b), x, info in zip(systems, xs, infos):
        _, rn = oracle.residual(A, b, host(x).reshape(b.shape))
        assert info["status"] == 0 and rn / np.linalg.norm(b) <= 1e-8
    # warm start from the converged x: nothing left to do
    infos2 = hz.solve_batched(ops, bs, xs, x0s=[x.clone() for x in xs])
    assert all(i["status"] == 0 and i["outer_iters"] == 0 for i in infos2)


def test_batched_barrier_timeout_is_reported_not_hung():
    import torch

    import paper_1811_03852_gb300 as hz

    systems = _systems([(64, 48, 20, 11, 12), (32, 24, 20, 13, 14)])
    ops = [hz.Operator(A) for A, _ in systems]
    bs = [dev(b.reshape(-1)) for _, b in systems]
    xs = [torch.empty(b.size, dtype=torch.float64, device="cuda") for _, b in systems]
    try:
        hz.batched_debug(timeout_ns=200_000_000, leave_block=1)
        st, infos = hz.solve_batched(ops, bs, xs, raise_on_error=False, strategy=hz.HZ_BATCH_PERSISTENT)
    finally:
        hz.batched_debug(0, -1)
    assert st == hz.HZ_ERR_TIMEOUT and all(i["status"] == hz.HZ_ERR_TIMEOUT for i in infos)
    # the context is still usable
    infos = hz.solve_batched(ops, bs, xs)
    assert all(i["status"] == 0 for i in infos)


def test_batched_rejects_bad_arguments():
    import torch

    import paper_1811_03852_gb300 as hz

    (A, b), = _systems([(8, 6, 5, 1, 2)])
    op = hz.Operator(A)
    bd = dev(b.reshape(-1))
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    st, _ = hz.solve_batched([op], [bd], [x], mode=hz.HZ_MODE_FP64, raise_on_error=False)
    assert st == hz.HZ_ERR_UNSUPPORTED
    st, _ = hz.solve_batched([op], [bd], [x], raise_on_error=False, strategy=3)
    assert st == hz.HZ_ERR_INVALID


@pytest.mark.parametrize("strategy", [1, 2])
def test_batched_strategies_match_single_solves(strategy):
    # persistent (1): same algorithm, its own launch shape (agrees to 1e-6);
    # sequential (2): each system through hz_solve (bit-identical to it)
    import torch

    import paper_1811_03852_gb300 as hz

    specs = [(96, 72, 20, 31, 32), (64, 48, 20, 33, 34), (130, 65, 11, 35, 36)]
    systems = _systems(specs, z_unit="m")
    xs, infos, ops = _batched(systems, strategy=strategy)
    for (A, b), x, info, op in zip(systems, xs, infos, ops):
        assert info["status"] == 0, info
        xd = torch.empty(b.size, dtype=torch.float64, device="cuda")
        single = op.solve(dev(b), xd)
        xsgl = host(xd).reshape(b.shape)
        if strategy == hz.HZ_BATCH_SEQUENTIAL:
            assert np.array_equal(x, xsgl) and info["inner_iters"] == single["inner_iters"]
        else:
            assert np.linalg.norm(x - xsgl) / np.linalg.norm(xsgl) <= 1e-6


@pytest.mark.parametrize("strategy", [0, 1])
def test_batched_32_uneven_systems_full_size(strategy):
    # the 32-system batch (grids 192x144, 320x240, 640x480, 70 levels): every
    # system's true residual recomputed by the oracle over all points, with the
    # automatic strategy (sequential at these sizes) and the persistent launch
    specs = [gen.batched_spec(i) for i in range(32)]
    specs = [(s["nx"], s["ny"], s["nz"], s["seed_coef"], s["seed_rhs"]) for s in specs]
    systems = _systems(specs, z_unit="radius")
    xs, infos, _ = _batched(systems, strategy=strategy)
    for (A, b), x, info in zip(systems, xs, infos):
        assert info["status"] == 0, info
        _, rn = oracle.residual(A, b, x)
        assert rn / np.linalg.norm(b) <= 1e-8


@pytest.mark.parametrize("strategy", [1, 2])
def test_many_right_hand_sides_of_one_operator(strategy):
    # one operator named several times (its extra right-hand sides get their own
    # work vectors), next to another operator twice: every solve reaches 1e-8
    # and matches its single solve
    import torch

    import paper_1811_03852_gb300 as hz

    A1 = gen.make_operator(48, 36, 20, 41, z_unit="m")
    A2 = gen.make_operator(40, 30, 12, 42, z_unit="m")
    op1, op2 = hz.Operator(A1), hz.Operator(A2)
    ops, As, bs = [], [], []
    for q in range(9):
        A, op, dims = (A1, op1, (48, 36, 20)) if q % 3 else (A2, op2, (40, 30, 12))
        ops.append(op)
        As.append(A)
        bs.append(gen.make_rhs(*dims, 500 + q))
    xs = [torch.empty(b.size, dtype=torch.float64, device="cuda") for b in bs]
    infos = hz.solve_batched(ops, [dev(b.reshape(-1)) for b in bs], xs, strategy=strategy)
    for A, b, x, info, op in zip(As, bs, xs, infos, ops):
        assert info["status"] == 0, info
        xh = host(x).reshape(b.shape)
        _, rn = oracle.residual(A, b, xh)
        assert rn / np.linalg.norm(b) <= 1e-8
        xd = torch.empty(b.size, dtype=torch.float64, device="cuda")
        op.solve(dev(b), xd)
        assert np.linalg.norm(xh - host(xd).reshape(b.shape)) / np.linalg.norm(xh) <= 1e-6


def test_persistent_solve_is_one_launch_and_replays_from_a_graph():
    # the whole batched solve is one cooperative launch; with use_graph it is
    # captured once and replayed on the next call with the same systems, with
    # the same bits as a direct launch
    import torch

    import paper_1811_03852_gb300 as hz

    specs = [(48, 36, 20, 61 + 2 * i, 62 + 2 * i) for i in range(6)]
    systems = _systems(specs, z_unit="m")
    ops = [hz.Operator(A) for A, _ in systems]
    bs = [dev(b.reshape(-1)) for _, b in systems]
    outs = []
    for use_graph in (0, 1, 1):  # direct, captured, replayed
        xs = [torch.full((b.numel(),), np.nan, dtype=torch.float64, device="cuda") for b in bs]
        infos = hz.solve_batched(ops, bs, xs, strategy=hz.HZ_BATCH_PERSISTENT, use_graph=use_graph)
        assert all(i["status"] == 0 and i["kernel_launches"] == 1 for i in infos), infos
        outs.append(([host(x) for x in xs], [i["inner_iters"] for i in infos]))
    for xs, its in outs[1:]:
        assert its == outs[0][1]
        assert all(np.array_equal(a, b) for a, b in zip(xs, outs[0][0]))
    for (A, b), x in zip(systems, outs[2][0]):
        _, rn = oracle.residual(A, b, x.reshape(b.shape))
        assert rn / np.linalg.norm(b) <= 1e-8


def test_small_systems_go_to_the_persistent_launch():
    # systems too small to fill the GPU alone: the automatic strategy is the
    # persistent launch (one launch for all of them)
    import paper_1811_03852_gb300 as hz

    systems = _systems([(48, 36, 70, 71 + 2 * i, 72 + 2 * i) for i in range(16)], z_unit="radius")
    xs, infos, _ = _batched(systems)
    for (A, b), x, info in zip(systems, xs, infos):
        assert info["status"] == 0 and info["kernel_launches"] == 1, info
        _, rn = oracle.residual(A, b, x)
        assert rn / np.linalg.norm(b) <= 1e-8
    del hz


def test_columns_per_thread_setting():
    # both launch shapes of the persistent kernel solve the batch; 4 columns per
    # thread with an nx that is not a multiple of 4 and unknown widths are refused
    import paper_1811_03852_gb300 as hz

    systems = _systems([(48, 36, 20, 71, 72), (40, 30, 20, 73, 74)], z_unit="m")
    try:
        for vec in (1, 4):
            hz.batched_set_vec(vec)
            xs, infos, _ = _batched(systems, strategy=hz.HZ_BATCH_PERSISTENT)
            for (A, b), x, info in zip(systems, xs, infos):
                assert info["status"] == 0 and info["kernel_launches"] == 1, info
                _, rn = oracle.residual(A, b, x)
                assert rn / np.linalg.norm(b) <= 1e-8
        odd = _systems([(38, 20, 10, 75, 76)], z_unit="m")
        with pytest.raises(hz.HzError):
            _batched(odd, strategy=hz.HZ_BATCH_PERSISTENT)
        for bad in (2, 3, -1, 8):
            with pytest.raises(hz.HzError):
                hz.batched_set_vec(bad)
    finally:
        hz.batched_set_vec(0)
