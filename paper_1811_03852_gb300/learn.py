"""Training and evaluation of the learned preconditioner stage (orchestration only).

Every numerical step runs in the CUDA library: the systems are solved by
hz_solve, the (residual, error) pairs are formed by hz_nn_make_pair, crops
are cut by hz_nn_crops, and the network is trained by hz_nn_train_step.
This module only decides which seeds, iterates and crop corners to use.

Data (one reading of the recipe): for each training system, the exact
solution x* comes from an FP64 solve to 1e-11; the plain mixed solver is run
for k = 1, 2, 4, ... inner iterations from x = 0 and each iterate x_k gives a
pair (stage input e1/sigma, target (x* - x_k - T^-1 r)/sigma).  Random
crops of crop x crop columns (all levels) plus a halo of 4 (the receptive
field of four 3x3x3 layers) are cut from every pair; the loss covers the
interior only, so each crop sees exactly the neighbourhood it would see in
the full field.  Crop corners are drawn from the counter-based generator in
``gen`` (they are inputs, not library arithmetic).
"""
from __future__ import annotations

import time

import numpy as np

HALO = 4


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
    """Train on the given (seed_coef, seed_rhs) systems.  Returns the list of losses."""
    torch = _torch()
    import gen
    import paper_1811_03852_gb300 as hz

    nx, ny, nz = dims
    cx = cy = crop + 2 * HALO
    bin_ = torch.empty(batch * cx * cy * nz, dtype=torch.float32, device="cuda")
    btg = torch.empty_like(bin_)
    losses = []
    steps_per_sys = max(1, steps // max(1, len(systems)))
    ctr = 0
    for si, (sc, sr) in enumerate(systems):
        A = gen.make_operator(nx, ny, nz, sc, z_unit=z_unit)
        b = torch.from_numpy(gen.make_rhs(nx, ny, nz, sr).reshape(-1)).cuda()
        op = hz.Operator(A)
        pairs = system_pairs(op, b, **({"iters": iters} if iters else {}))
        del op
        for _ in range(steps_per_sys):
            # one pair per step, `batch` crops of it, stacked along j by the crop kernel
            pi = min(int(gen.uniform(seed, 11, ctr) * len(pairs)), len(pairs) - 1)
            ctr += 1
            corners = []
            for q in range(batch):
                i0 = int(gen.uniform(seed, 12, ctr) * nx)
                j0 = int(gen.uniform(seed, 13, ctr) * max(1, ny - crop))
                ctr += 1
                corners.append((i0 - HALO, j0 - HALO))
            hz.nn_crops(pairs[pi][0], pairs[pi][1], dims, corners, cx, cy, bin_, btg)
            loss = net.train_step(bin_, btg, (cx, batch * cy, nz), lr=lr, seg_ny=cy, periodic=False, border=HALO,
                                  clip=clip)
            losses.append(loss)
            if log and len(losses) % 20 == 0:
                log(f"step {len(losses)} system {si} loss {loss:.4f}")
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
