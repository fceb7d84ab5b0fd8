"""Pins for the conv-net oracle (oracle/nn.py): library routines, autograd, adjoint identity, finite differences."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import gen
from oracle import nn as onn


def _rand(shape, seed, scale=1.0):
    return scale * gen.normals(seed, 3, int(np.prod(shape))).reshape(shape)


def _params(seed):
    ps = []
    for li in range(4):
        ci, co = onn.CHANNELS[li], onn.CHANNELS[li + 1]
        ps.append((_rand((co, ci, 3, 3, 3), seed + li, 1.0 / np.sqrt(27 * ci)), _rand((co,), seed + 10 + li, 0.1)))
    return ps


def _torch_pad(x, periodic):
    # x: (N, C, nz, ny, nx); pad i (last dim) circularly or with zeros, then j and k with zeros
    if periodic:
        x = F.pad(x, (1, 1, 0, 0, 0, 0), mode="circular")
    else:
        x = F.pad(x, (1, 1, 0, 0, 0, 0))
    return F.pad(x, (0, 0, 1, 1, 1, 1))


def _torch_net(params, x, periodic):
    h = x
    for li, (W, b) in enumerate(params):
        z = F.conv3d(_torch_pad(h, periodic), W, b)
        h = F.gelu(z) if li < 3 else z
    return h


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("cin,cout", [(1, 16), (16, 16), (16, 1), (3, 2)])
def test_conv_matches_torch_conv3d(periodic, cin, cout):
    x = _rand((cin, 5, 6, 7), 1)
    W = _rand((cout, cin, 3, 3, 3), 2)
    b = _rand((cout,), 3)
    y = onn.conv3d(x, W, b, periodic)
    ref = F.conv3d(_torch_pad(torch.from_numpy(x)[None], periodic), torch.from_numpy(W), torch.from_numpy(b))[0]
    assert np.allclose(y, ref.numpy(), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("periodic", [True, False])
def test_conv_adjoint_identity(periodic):
    x = _rand((4, 5, 6, 7), 4)
    dy = _rand((3, 5, 6, 7), 5)
    W = _rand((3, 4, 3, 3, 3), 6)
    lhs = np.sum((onn.conv3d(x, W, np.zeros(3), periodic)) * dy)
    rhs = np.sum(x * onn.conv3d_input_grad(dy, W, periodic))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_gelu_and_derivative():
    z = np.linspace(-6, 6, 1001)
    assert np.allclose(onn.gelu(z), F.gelu(torch.from_numpy(z), approximate="none").numpy(), rtol=1e-14, atol=1e-15)
    h = 1e-6
    fd = (onn.gelu(z + h) - onn.gelu(z - h)) / (2 * h)
    assert np.allclose(onn.gelu_grad(z), fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("periodic", [True, False])
def test_network_gradients_match_autograd(periodic):
    params = _params(20)
    x = _rand((1, 4, 5, 6), 30)
    t = _rand((1, 4, 5, 6), 31)
    y, cache = onn.forward(params, x, periodic)
    loss, dy = onn.rel_mse(y, t)
    grads = onn.backward(params, cache, dy, periodic)
    tp = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in params]
    ty = _torch_net(tp, torch.from_numpy(x)[None], periodic)[0]
    tt = torch.from_numpy(t)
    tl = torch.sum((ty - tt) ** 2) / torch.sum(tt ** 2)
    tl.backward()
    assert np.allclose(y, ty.detach().numpy(), rtol=1e-12, atol=1e-12)
    assert abs(loss - tl.item()) <= 1e-12 * loss
    for (dW, db), (W, b) in zip(grads, tp):
        assert np.allclose(dW, W.grad.numpy(), rtol=1e-10, atol=1e-13)
        assert np.allclose(db, b.grad.numpy(), rtol=1e-10, atol=1e-13)


def test_network_gradient_finite_differences():
    params = _params(40)
    x = _rand((1, 3, 4, 5), 41)
    t = _rand((1, 3, 4, 5), 42)
    flat = onn.flatten(params)

    def loss_of(f):
        y, _ = onn.forward(onn.unflatten(f), x)
        return onn.rel_mse(y, t)[0]

    y, cache = onn.forward(params, x)
    _, dy = onn.rel_mse(y, t)
    g = onn.flatten([(dW, db) for dW, db in onn.backward(params, cache, dy)])
    rng = np.random.default_rng(0)
    for idx in rng.choice(flat.size, 25, replace=False):
        e = np.zeros_like(flat)
        e[idx] = 1e-6
        fd = (loss_of(flat + e) - loss_of(flat - e)) / 2e-6
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])), (idx, fd, g[idx])


def test_masked_loss_ignores_outside_points():
    y = _rand((1, 2, 3, 4), 50)
    t = _rand((1, 2, 3, 4), 51)
    mask = np.zeros_like(t, dtype=bool)
    mask[:, :, 1:, 1:3] = True
    L, dy = onn.rel_mse(y, t, mask)
    assert np.all(dy[~mask] == 0)
    assert abs(L - np.sum((y - t)[mask] ** 2) / np.sum(t[mask] ** 2)) <= 1e-14


def test_adam_matches_torch():
    w = _rand((50,), 60)
    m = np.zeros(50)
    v = np.zeros(50)
    tw = torch.tensor(w, requires_grad=True)
    opt = torch.optim.Adam([tw], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = _rand((50,), 70 + step)
        w, m, v = onn.adam_step(w, g, m, v, step)
        opt.zero_grad()
        tw.grad = torch.from_numpy(g)
        opt.step()
        assert np.allclose(w, tw.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_param_count_and_flat_layout():
    assert onn.num_params() == (16 * 27 + 16) + 2 * (16 * 16 * 27 + 16) + (16 * 27 + 1)
    p = _params(80)
    assert all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
               for a, b in zip(p, onn.unflatten(onn.flatten(p))))


def _crop_bands(nz, ny, nx, seed):
    import oracle

    A = gen.make_operator(nx, ny, nz, seed, z_unit="m")
    return oracle.scale(A)


def test_crop_operator_matches_dense_assembly_and_its_transpose():
    # on one crop (no stacking) Ahat with absent neighbours outside is I + bands
    # with the periodic couplings removed: compare with a dense assembly; the
    # transpose is the dense transpose
    from conftest import dense_from_hat

    nz, ny, nx = 3, 4, 5
    Ah = _crop_bands(nz, ny, nx, 7)
    Ah[0][:, :, -1] = 0.0  # E of the last column and W of the first would wrap: a crop has no wrap
    Ah[1][:, :, 0] = 0.0
    M = dense_from_hat(Ah)
    d = np.random.default_rng(1).standard_normal((nz, ny, nx))
    assert np.allclose(onn.ahat_crop(Ah, d).ravel(), M @ d.ravel(), rtol=1e-13, atol=1e-13)
    assert np.allclose(onn.ahat_crop_transpose(Ah, d).ravel(), M.T @ d.ravel(), rtol=1e-13, atol=1e-13)


def test_crop_operator_segments_do_not_couple():
    # stacked crops: rows of one segment never see the next segment's
    nz, ny, nx, seg = 2, 8, 5, 4
    Ah = _crop_bands(nz, ny, nx, 8)
    d = np.zeros((nz, ny, nx))
    d[:, :seg] = np.random.default_rng(2).standard_normal((nz, seg, nx))
    y = onn.ahat_crop(Ah, d, seg)
    assert np.all(y[:, seg:] == 0.0)
    yt = onn.ahat_crop_transpose(Ah, d, seg)
    assert np.all(yt[:, seg:] == 0.0)


def test_op_loss_gradient_finite_differences_and_autograd():
    import torch

    nz, ny, nx, seg = 3, 12, 9, 6
    rng = np.random.default_rng(3)
    Ah = _crop_bands(nz, ny, nx, 9)
    y = rng.standard_normal((nz, ny, nx))
    t = rng.standard_normal((nz, ny, nx))
    mask = np.zeros((nz, ny, nx), dtype=bool)
    for s in range(0, ny, seg):
        mask[:, s + 2:s + seg - 2, 2:nx - 2] = True
    loss, g = onn.op_loss(y, t, Ah, mask, seg)
    # autograd of the same expression assembled from dense per-segment matrices
    from conftest import dense_from_hat

    yt = torch.tensor(y, requires_grad=True)
    tt = torch.tensor(t)
    mk = torch.tensor(mask)
    u_parts, a_parts = [], []
    for s in range(0, ny, seg):
        B = Ah[:, :, s:s + seg, :].copy()
        B[0][:, :, -1] = 0.0
        B[1][:, :, 0] = 0.0
        B[2][:, -1, :] = 0.0  # N of the segment's last row, S of its first: outside the segment
        B[3][:, 0, :] = 0.0
        M = torch.tensor(dense_from_hat(B))
        u_parts.append(torch.where(mk[:, s:s + seg].reshape(-1), M @ (yt[:, s:s + seg] - tt[:, s:s + seg]).reshape(-1), 0.0))
        a_parts.append(torch.where(mk[:, s:s + seg].reshape(-1), M @ tt[:, s:s + seg].reshape(-1), 0.0))
    u = torch.cat(u_parts)
    a = torch.cat(a_parts)
    L = (u * u).sum() / (a * a).sum()
    L.backward()
    assert abs(float(L) - loss) <= 1e-12 * abs(loss)
    assert np.allclose(yt.grad.numpy(), g, rtol=1e-10, atol=1e-12)
    # and a central finite difference in one coordinate
    e = np.zeros_like(y)
    e[1, 4, 3] = 1e-6
    lp, _ = onn.op_loss(y + e, t, Ah, mask, seg)
    lm, _ = onn.op_loss(y - e, t, Ah, mask, seg)
    assert abs((lp - lm) / 2e-6 - g[1, 4, 3]) <= 1e-6 * max(1.0, abs(g[1, 4, 3]))
