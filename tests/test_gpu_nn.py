"""Learned preconditioner stage on the GPU against the FP64 conv-net oracle.

Bars: layer by layer (each GPU layer fed the GPU's own BF16 inputs and the
BF16-rounded weights, so only FP32 accumulation differs) <= 1e-4 relative in
the 2-norm; the whole BF16 network against the all-FP64 oracle <= 2e-2 rel-L2;
gradients layer by layer <= 1e-3 rel-L2; Adam <= 1e-6.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_util import dev, host
from oracle import nn as onn

pytestmark = pytest.mark.gpu


def bf16(a):
    import torch

    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def rand_params(seed, scale=1.0):
    ps = []
    for li in range(4):
        ci, co = onn.CHANNELS[li], onn.CHANNELS[li + 1]
        W = gen.normals(seed + li, 5, co * ci * 27).reshape(co, ci, 3, 3, 3) * scale / np.sqrt(27 * ci)
        b = 0.1 * gen.normals(seed + 10 + li, 5, co)
        ps.append((W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)))
    return ps


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def _net(params):
    import paper_1811_03852_gb300 as hz

    return hz.Net(onn.flatten(params).astype(np.float32))


def _rounded(params):
    return [(bf16(W), bf16(b)) for W, b in params]


DIMS = [((20, 12, 6), 12, True), ((37, 9, 5), 9, True), ((24, 12, 4), 6, False), ((16, 16, 3), 16, False),
        # rows of 128 points and more: the tensor-core (tcgen05) 16->16 and 16->1 layers, ragged
        # tiles in i, crop seams every 4 rows, a single odd segment, one level
        ((160, 12, 6), 12, True), ((136, 8, 4), 4, False), ((129, 5, 3), 5, True), ((256, 6, 1), 6, True)]


@pytest.mark.parametrize("dims,seg,periodic", DIMS)
def test_forward_layerwise_and_end_to_end(dims, seg, periodic):
    import torch

    nx, ny, nz = dims
    n = nx * ny * nz
    params = rand_params(7)
    net = _net(params)
    x = gen.normals(8, 0, n).astype(np.float32).reshape(nz, ny, nx)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    z = torch.empty(3 * n * 16, dtype=torch.float32, device="cuda")
    net.forward(dev(x), y, dims, seg_ny=seg, periodic=periodic, zout=z)
    yg = host(y).reshape(nz, ny, nx)
    zg = [host(z)[q * n * 16:(q + 1) * n * 16].reshape(nz, ny, nx, 16).transpose(3, 0, 1, 2) for q in range(3)]
    P = _rounded(params)

    # stacked crops are independent: run the oracle per crop
    def per_crop(fn, a):
        outs = [fn(a[:, :, s * seg:(s + 1) * seg, :]) for s in range(ny // seg)]
        return np.concatenate(outs, axis=2)

    h_in = x[None].astype(np.float64)
    for li in range(3):
        W, b = P[li]
        zo = per_crop(lambda a: onn.conv3d(a, W, b, periodic), h_in)
        assert rel(zg[li], zo) <= 1e-4, (li, rel(zg[li], zo))
        h_in = bf16(onn.gelu(zg[li]))
    W, b = P[3]
    yo = per_crop(lambda a: onn.conv3d(a, W, b, periodic), h_in)[0]
    assert rel(yg, yo) <= 1e-4
    # the whole BF16 network against the FP64 oracle
    yf = per_crop(lambda a: onn.forward(params, a, periodic)[0], x[None].astype(np.float64))[0]
    assert rel(yg, yf) <= 2e-2, rel(yg, yf)


@pytest.mark.parametrize("dims,seg,periodic", DIMS[:3] + [DIMS[5]])
def test_gradient_layerwise(dims, seg, periodic):
    import torch

    nx, ny, nz = dims
    n = nx * ny * nz
    border = 1 if not periodic else 0
    params = rand_params(17)
    net = _net(params)
    x = gen.normals(18, 0, n).astype(np.float32).reshape(nz, ny, nx)
    t = gen.normals(19, 0, n).astype(np.float32).reshape(nz, ny, nx)
    g, loss = net.gradient(dev(x), dev(t), dims, seg_ny=seg, periodic=periodic, border=border)
    # reconstruct the GPU's activations and run the oracle backward on them
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    z = torch.empty(3 * n * 16, dtype=torch.float32, device="cuda")
    net.forward(dev(x), y, dims, seg_ny=seg, periodic=periodic, zout=z)
    yg = host(y).reshape(1, nz, ny, nx).astype(np.float64)
    zg = [host(z)[q * n * 16:(q + 1) * n * 16].reshape(nz, ny, nx, 16).transpose(3, 0, 1, 2) for q in range(3)]
    P = _rounded(params)
    mask = np.zeros((1, nz, ny, nx), dtype=bool)
    for s in range(ny // seg):
        mask[:, :, s * seg + border:(s + 1) * seg - border, border:nx - border] = True
    lo, dy = onn.rel_mse(yg, t[None].astype(np.float64), mask)
    assert abs(loss - lo) <= 1e-5 * lo
    hs = [x[None].astype(np.float64)] + [bf16(onn.gelu(zz)) for zz in zg]

    def crops_sum(fn, *arrs):
        tot = None
        for s in range(ny // seg):
            r = fn(*[a[:, :, s * seg:(s + 1) * seg, :] for a in arrs])
            tot = r if tot is None else tuple(u + v for u, v in zip(tot, r))
        return tot

    def crops_cat(fn, *arrs):
        return np.concatenate([fn(*[a[:, :, s * seg:(s + 1) * seg, :] for a in arrs]) for s in range(ny // seg)], axis=2)

    grads = [None] * 4
    gcur = dy
    for li in range(3, -1, -1):
        if li < 3:
            gcur = gcur * onn.gelu_grad(zg[li])
        grads[li] = crops_sum(lambda h, d: onn.conv3d_weight_grad(h, d, periodic), hs[li], gcur)
        if li > 0:
            W = P[li][0]
            gcur = crops_cat(lambda d: onn.conv3d_input_grad(d, W, periodic), gcur)
    gref = onn.flatten(grads)
    o = 0
    for li in range(4):
        ci, co = onn.CHANNELS[li], onn.CHANNELS[li + 1]
        k = co * ci * 27 + co
        assert rel(g[o:o + k], gref[o:o + k]) <= 1e-3, (li, rel(g[o:o + k], gref[o:o + k]))
        o += k


def test_adam_step_and_training_progress():
    import torch

    nx, ny, nz, seg = 16, 16, 4, 8
    n = nx * ny * nz
    params = rand_params(27)
    net = _net(params)
    x = dev(gen.normals(28, 0, n).astype(np.float32))
    # a target the network can approach: a smoothed copy of the input
    xs = gen.normals(28, 0, n).reshape(nz, ny, nx)
    t = dev((0.5 * xs + 0.25 * (np.roll(xs, 1, 2) + np.roll(xs, -1, 2))).astype(np.float32))
    g, _ = net.gradient(x, t, (nx, ny, nz), seg_ny=seg, border=1)
    w0 = net.get_params().astype(np.float64)
    net2 = _net(params)
    net2.train_step(x, t, (nx, ny, nz), lr=1e-3, seg_ny=seg, border=1)
    w1 = net2.get_params().astype(np.float64)
    w_ref, _, _ = onn.adam_step(w0, g, np.zeros_like(w0), np.zeros_like(w0), 1)
    assert np.max(np.abs(w1 - w_ref)) <= 1e-6 * max(1.0, np.max(np.abs(w_ref)))
    losses = [net2.train_step(x, t, (nx, ny, nz), lr=3e-3, seg_ny=seg, border=1) for _ in range(60)]
    assert losses[-1] < 0.7 * losses[0], losses[::10]


def test_save_load_roundtrip(tmp_path):
    params = rand_params(37)
    net = _net(params)
    p = tmp_path / "nn.bin"
    net.save(p)
    import paper_1811_03852_gb300 as hz

    other = hz.Net()
    other.load(p)
    assert np.array_equal(other.get_params(), net.get_params())


def test_crops_match_numpy_indexing():
    import torch

    import paper_1811_03852_gb300 as hz

    nx, ny, nz = 30, 20, 3
    fa = gen.normals(1, 1, nx * ny * nz).astype(np.float32).reshape(nz, ny, nx)
    fb = gen.normals(2, 1, nx * ny * nz).astype(np.float32).reshape(nz, ny, nx)
    corners = [(26, -2), (0, 5), (13, 16)]
    cx, cy = 8, 6
    oa = torch.empty(len(corners) * cx * cy * nz, dtype=torch.float32, device="cuda")
    ob = torch.empty_like(oa)
    hz.nn_crops(dev(fa), dev(fb), (nx, ny, nz), corners, cx, cy, oa, ob)
    ga = host(oa).reshape(nz, len(corners) * cy, cx)
    for q, (i0, j0) in enumerate(corners):
        for jj in range(cy):
            j = j0 + jj
            want = fa[:, j, [(i0 + ii) % nx for ii in range(cx)]] if 0 <= j < ny else np.zeros((nz, cx))
            assert np.array_equal(ga[:, q * cy + jj, :], want)


def test_make_pair_matches_oracle():
    import torch

    import paper_1811_03852_gb300 as hz

    nx, ny, nz = 24, 16, 10
    A, b = gen.make_system(nx, ny, nz, 3, 4, z_unit="m")
    xs, _ = oracle.solve(A, b, mode=oracle.MODE_FP64, tol=1e-12, eta=1e-13)
    xk = 0.5 * xs + 0.1 * gen.normals(5, 2, xs.size).reshape(xs.shape)
    op = hz.Operator(A)
    n = xs.size
    inp = torch.empty(n, dtype=torch.float32, device="cuda")
    tg = torch.empty(n, dtype=torch.float32, device="cuda")
    sig = op.make_pair(dev(b), dev(xk), dev(xs), inp, tg)
    Ah = oracle.scale(A)
    r = oracle.residual(A, b, xk)[0] / A[0]
    z1 = oracle.apply_Tinv(Ah, r)
    e1 = r - oracle.matvec_hat(Ah, z1)
    s = np.sqrt(np.mean(e1 ** 2))
    assert abs(sig - s) <= 1e-5 * s
    assert rel(host(inp).reshape(xs.shape), e1 / s) <= 1e-4
    assert rel(host(tg).reshape(xs.shape), (xs - xk - z1) / s) <= 1e-4


def _fgmres_nn(A, b, net, **kw):
    import torch

    import paper_1811_03852_gb300 as hz

    op = hz.Operator(A)
    if net is not None:
        op.set_nn(net)
    x = torch.empty(b.size, dtype=torch.float64, device="cuda")
    info = op.solve(dev(b), x, krylov=hz.HZ_KRYLOV_FGMRES, precond=hz.HZ_PRE_TRI_NN if net is not None else hz.HZ_PRE_TRI,
                    **kw)
    return host(x).reshape(b.shape), info


def test_zero_network_equals_plain_preconditioner():
    import paper_1811_03852_gb300 as hz

    A, b = gen.make_system(48, 24, 10, 5, 6, z_unit="m")
    net = hz.Net()  # all parameters zero: the stage adds nothing (z = z1 exactly)
    x1, i1 = _fgmres_nn(A, b, net)
    x0, i0 = _fgmres_nn(A, b, None)
    # same iterates; the stall test may still switch the (useless) stage off
    assert i1["status"] == 0 and i1["inner_iters"] == i0["inner_iters"]
    assert np.array_equal(x1, x0)


def test_bad_network_falls_back_and_still_converges():
    A, b = gen.make_system(48, 24, 10, 5, 6, z_unit="m")
    net = _net(rand_params(99, scale=30.0))  # large random weights: a harmful stage
    x, info = _fgmres_nn(A, b, net)
    assert info["status"] == 0 and info["fallbacks"] >= 1
    _, rn = oracle.residual(A, b, x)
    assert rn / np.linalg.norm(b) <= 1e-8


@pytest.mark.parametrize("dims,seg,border", [((24, 12, 4), 6, 2), ((136, 8, 4), 4, 1), ((40, 20, 7), 10, 3)])
def test_gradient_of_the_operator_weighted_loss(dims, seg, border):
    # the loss of the learned stage's training, ||mask Ahat (y - t)||^2 / ||mask Ahat t||^2,
    # and its gradient through the network, against the FP64 oracle on the GPU's
    # own activations (as in the test above)
    import torch

    nx, ny, nz = dims
    n = nx * ny * nz
    params = rand_params(23)
    net = _net(params)
    x = gen.normals(24, 0, n).astype(np.float32).reshape(nz, ny, nx)
    t = gen.normals(25, 0, n).astype(np.float32).reshape(nz, ny, nx)
    bands = oracle.scale(gen.make_operator(nx, ny, nz, 26, z_unit="m")).astype(np.float32)
    g, loss = net.gradient_op(dev(x), dev(t), dev(bands), dims, seg_ny=seg, border=border)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    z = torch.empty(3 * n * 16, dtype=torch.float32, device="cuda")
    net.forward(dev(x), y, dims, seg_ny=seg, periodic=False, zout=z)
    yg = host(y).reshape(nz, ny, nx).astype(np.float64)
    zg = [host(z)[q * n * 16:(q + 1) * n * 16].reshape(nz, ny, nx, 16).transpose(3, 0, 1, 2) for q in range(3)]
    P = _rounded(params)
    mask = np.zeros((nz, ny, nx), dtype=bool)
    for s in range(ny // seg):
        mask[:, s * seg + border:(s + 1) * seg - border, border:nx - border] = True
    lo, dy = onn.op_loss(yg, t.astype(np.float64), bands.astype(np.float64), mask, seg)
    assert abs(loss - lo) <= 1e-4 * lo, (loss, lo)
    dy = dy[None]
    hs = [x[None].astype(np.float64)] + [bf16(onn.gelu(zz)) for zz in zg]

    def crops_sum(fn, *arrs):
        tot = None
        for s in range(ny // seg):
            r = fn(*[a[:, :, s * seg:(s + 1) * seg, :] for a in arrs])
            tot = r if tot is None else tuple(u + v for u, v in zip(tot, r))
        return tot

    def crops_cat(fn, *arrs):
        return np.concatenate([fn(*[a[:, :, s * seg:(s + 1) * seg, :] for a in arrs]) for s in range(ny // seg)], axis=2)

    grads = [None] * 4
    gcur = dy
    for li in range(3, -1, -1):
        if li < 3:
            gcur = gcur * onn.gelu_grad(zg[li])
        grads[li] = crops_sum(lambda h, d: onn.conv3d_weight_grad(h, d, False), hs[li], gcur)
        if li > 0:
            W = P[li][0]
            gcur = crops_cat(lambda d: onn.conv3d_input_grad(d, W, False), gcur)
    gref = onn.flatten(grads)
    o = 0
    for li in range(4):
        ci, co = onn.CHANNELS[li], onn.CHANNELS[li + 1]
        k = co * ci * 27 + co
        assert rel(g[o:o + k], gref[o:o + k]) <= 1e-3, (li, rel(g[o:o + k], gref[o:o + k]))
        o += k
