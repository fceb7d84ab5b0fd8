"""Training and evaluation of the learned preconditioner stage (orchestration only).

Every numerical step runs in the CUDA library: hz_nn_train solves each
system (hz_solve), forms its (residual, error) pairs (hz_nn_make_pair), cuts
random crops (hz_nn_crops, corners from its own counter-based generator)
and takes the Adam steps (hz_nn_train_step).  This module only chooses the
seeds of the training and test systems and evaluates.

Data (one reading of the recipe): for each training system, the exact
solution x* comes from an FP64 solve to 1e-11; the plain mixed solver is run
for k = 1, 2, 4, ... inner iterations from x = 0 and each iterate x_k gives a
pair (stage input e1/sigma, target (x* - x_k - T^-1 r)/sigma).  Random
crops of crop x crop columns (all levels) plus a halo of 4 (the receptive
field of four 3x3x3 layers) are cut from every pair; the loss covers the
interior only, so each crop sees exactly the neighbourhood it would see in
the full field.
"""
from __future__ import annotations

import numpy as np


def _torch():
    import torch

    return torch


def init_params(seed: int, scale: float = 1.0) -> np.ndarray:
    """He-style initial parameters (flat, library layout) from seeded normals; last layer small."""
    import gen

    chans = (1, 16, 16, 16, 1)
    out = []
    for li in range(4):
        ci, co = chans[li], chans[li + 1]
        std = scale * np.sqrt(2.0 / (27 * ci)) * (0.1 if li == 3 else 1.0)
        out.append(std * gen.normals(seed + li, 9, co * ci * 27))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def system_pairs(op, b_dev, iters=(1, 2, 4, 8, 16, 32), eta_star=1e-11):
    """(input, target) device fields for the iterates x_k of one system, plus x*."""
    torch = _torch()
    import paper_1811_03852_gb300 as hz

    n = b_dev.numel()
    xs = torch.empty(n, dtype=torch.float64, device=b_dev.device)
    op.solve(b_dev, xs, mode=hz.HZ_MODE_FP64, tol=eta_star, raise_on_error=False)
    pairs = []
    xk = torch.empty_like(xs)
    for k in iters:
        info = op.solve(b_dev, xk, max_outer=1, max_inner=k, inner_tol=1e-12, raise_on_error=False)
        if info["inner_iters"] < 1:
            continue
        inp = torch.empty(n, dtype=torch.float32, device=b_dev.device)
        tg = torch.empty(n, dtype=torch.float32, device=b_dev.device)
        op.make_pair(b_dev, xk, xs, inp, tg)
        pairs.append((inp, tg))
    return pairs


def train(net, systems, dims, steps=200, batch=16, crop=64, lr=3e-4, seed=0, z_unit="radius", iters=None,
          log=None, clip=1.0):
    """Train on the given (seed_coef, seed_rhs) systems, one hz_nn_train call per system (the
    library forms the pairs, draws the crops and takes the Adam steps; the operator exists only
    for its call).  Returns the list of losses."""
    torch = _torch()
    import gen
    import paper_1811_03852_gb300 as hz

    nx, ny, nz = dims
    losses = []
    steps_per_sys = max(1, steps // max(1, len(systems)))
    for si, (sc, sr) in enumerate(systems):
        A = gen.make_operator(nx, ny, nz, sc, z_unit=z_unit)
        b = torch.from_numpy(gen.make_rhs(nx, ny, nz, sr).reshape(-1)).cuda()
        op = hz.Operator(A)
        kw = {"iterates": iters} if iters else {}
        losses += net.train(op, b, steps=steps_per_sys, batch=batch, crop=crop, lr=lr, clip=clip, seed=seed,
                            stream=si, **kw)
        op.close()
        if log:
            log(f"system {si} ({sc}/{sr}): {len(losses)} steps, last loss {losses[-1]:.4f}")
    return losses


def evaluate(net, systems, dims, z_unit="radius", m=30):
    """Plain vs learned FGMRES(m) on the given systems: per-system inner iterations, seconds, status, fallbacks."""
    torch = _torch()
    import gen
    import paper_1811_03852_gb300 as hz

    nx, ny, nz = dims
    rows = []
    for sc, sr in systems:
        A = gen.make_operator(nx, ny, nz, sc, z_unit=z_unit)
        b = torch.from_numpy(gen.make_rhs(nx, ny, nz, sr).reshape(-1)).cuda()
        op = hz.Operator(A)
        x = torch.empty_like(b)
        plain = op.solve(b, x, krylov=hz.HZ_KRYLOV_FGMRES, fgmres_m=m, raise_on_error=False)
        op.set_nn(net)
        learned = op.solve(b, x, krylov=hz.HZ_KRYLOV_FGMRES, fgmres_m=m, precond=hz.HZ_PRE_TRI_NN,
                           raise_on_error=False)
        rows.append({"plain": plain, "learned": learned})
    return rows
