"""Learned preconditioner end to end (GPU): train on a few systems, evaluate on held-out ones.

Shows what the trained stage gains over plain T^-1 inside the same FGMRES
solver (printed), and checks that every learned solve still reaches the true
FP64 residual 1e-8 (recomputed by the oracle) and is never much worse than the
plain one (the stall fallback bounds the loss).
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("z_unit", ["m", "radius"])
def test_train_then_solve_held_out(z_unit):
    import torch

    import paper_1811_03852_gb300 as hz
    from paper_1811_03852_gb300 import learn

    dims = (64, 48, 20)
    net = hz.Net(learn.init_params(5))
    train_sys = [(300 + 2 * i, 301 + 2 * i) for i in range(6)]
    test_sys = [(400 + 2 * i, 401 + 2 * i) for i in range(3)]
    losses = learn.train(net, train_sys, dims, steps=120, batch=8, crop=24, lr=1e-3, seed=3, z_unit=z_unit,
                         iters=(1, 2, 4, 8, 16))
    assert np.isfinite(losses).all()
    if z_unit == "m":  # on the easy family T^-1 leaves almost nothing to learn
        assert np.mean(losses[-10:]) < np.mean(losses[:10])
    rows = learn.evaluate(net, test_sys, dims, z_unit=z_unit)
    gains = []
    for (sc, sr), row in zip(test_sys, rows):
        p, l = row["plain"], row["learned"]
        assert p["status"] == 0 and l["status"] == 0
        assert l["inner_iters"] <= 1.5 * p["inner_iters"] + 10
        gains.append(p["inner_iters"] / max(1, l["inner_iters"]))
        # the learned solve's x is correct: recompute its residual
        A = gen.make_operator(*dims, sc, z_unit=z_unit)
        b = gen.make_rhs(*dims, sr)
        op = hz.Operator(A)
        op.set_nn(net)
        x = torch.empty(b.size, dtype=torch.float64, device="cuda")
        op.solve(torch.from_numpy(b.reshape(-1)).cuda(), x, krylov=hz.HZ_KRYLOV_FGMRES, precond=hz.HZ_PRE_TRI_NN)
        _, rn = oracle.residual(A, b, x.cpu().numpy().reshape(b.shape))
        assert rn / np.linalg.norm(b) <= 1e-8
    print(f"\n[{z_unit}] loss {losses[0]:.3f} -> {np.mean(losses[-10:]):.3f}; plain/learned FGMRES iterations per "
          f"held-out system: {[round(g, 2) for g in gains]} (>1 = the learned stage saves iterations); "
          f"details: {[(r['plain']['inner_iters'], r['learned']['inner_iters'], r['learned']['fallbacks']) for r in rows]}")
