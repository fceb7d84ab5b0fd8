"""FP64 NumPy reference of the learned preconditioner stage -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and the benchmark's CPU-baseline leg may import
this module; the GPU library shares no code with it.

Network (the learned stage of the flexible solver): four 3-D convolutions,
channels 1 -> 16 -> 16 -> 16 -> 1, each kernel 3 (levels) x 3 (latitude) x 3
(longitude), exact-erf GELU after the first three.  A convolution here is a
cross-correlation with a bias:

    y[o, k, j, i] = b[o] + sum_{c, dk, dj, di} W[o, c, dk+1, dj+1, di+1] * x[c, k+dk, j+dj, i+di]

for dk, dj, di in {-1, 0, 1}.  Outside the grid in k (levels) and j (latitude)
x is zero; in i (longitude) it wraps around when ``periodic`` (full fields) and
is zero otherwise (training crops).

Arrays: activations (C, nz, ny, nx); weights (Cout, Cin, 3, 3, 3); biases (Cout,).
Pinned in tests/test_oracle_nn.py against torch.nn.functional.conv3d on
explicitly padded inputs, torch autograd, finite differences, the adjoint
identity <conv x, y> = <x, conv^T y>, and torch.optim.Adam.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

CHANNELS = (1, 16, 16, 16, 1)
TAPS = [(dk, dj, di) for dk in (-1, 0, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]


def _pad(x, periodic):
    """Pad (C, nz, ny, nx) by one: zeros in k and j, wrap (or zeros) in i."""
    C, nz, ny, nx = x.shape
    xp = np.zeros((C, nz + 2, ny + 2, nx + 2), dtype=x.dtype)
    xp[:, 1:-1, 1:-1, 1:-1] = x
    if periodic:
        xp[:, 1:-1, 1:-1, 0] = x[:, :, :, -1]
        xp[:, 1:-1, 1:-1, -1] = x[:, :, :, 0]
    return xp


def conv3d(x, W, b, periodic=True):
    """The convolution defined above: (Cin, nz, ny, nx) -> (Cout, nz, ny, nx)."""
    C, nz, ny, nx = x.shape
    xp = _pad(x, periodic)
    y = np.zeros((W.shape[0], nz, ny, nx))
    for dk, dj, di in TAPS:
        xs = xp[:, 1 + dk:1 + dk + nz, 1 + dj:1 + dj + ny, 1 + di:1 + di + nx]
        y += np.einsum("oc,czyx->ozyx", W[:, :, dk + 1, dj + 1, di + 1], xs)
    return y + b[:, None, None, None]


def conv3d_input_grad(dy, W, periodic=True):
    """Adjoint of conv3d with respect to its input: dx = conv^T dy."""
    O, nz, ny, nx = dy.shape
    C = W.shape[1]
    dxp = np.zeros((C, nz + 2, ny + 2, nx + 2))
    for dk, dj, di in TAPS:
        dxp[:, 1 + dk:1 + dk + nz, 1 + dj:1 + dj + ny, 1 + di:1 + di + nx] += np.einsum(
            "oc,ozyx->czyx", W[:, :, dk + 1, dj + 1, di + 1], dy)
    dx = dxp[:, 1:-1, 1:-1, 1:-1].copy()
    if periodic:  # contributions that left through the longitude seam re-enter on the other side
        dx[:, :, :, -1] += dxp[:, 1:-1, 1:-1, 0]
        dx[:, :, :, 0] += dxp[:, 1:-1, 1:-1, -1]
    return dx


def conv3d_weight_grad(x, dy, periodic=True):
    """dW[o, c, tap] = sum_p dy[o, p] x[c, p + tap], db[o] = sum_p dy[o, p]."""
    C, nz, ny, nx = x.shape
    xp = _pad(x, periodic)
    dW = np.zeros((dy.shape[0], C, 3, 3, 3))
    for dk, dj, di in TAPS:
        xs = xp[:, 1 + dk:1 + dk + nz, 1 + dj:1 + dj + ny, 1 + di:1 + di + nx]
        dW[:, :, dk + 1, dj + 1, di + 1] = np.einsum("ozyx,czyx->oc", dy, xs)
    return dW, dy.sum(axis=(1, 2, 3))


def gelu(z):
    """GELU with the exact normal CDF: z * Phi(z)."""
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d/dz [z Phi(z)] = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, x, periodic=True):
    """params: list of 4 (W, b).  x: (1, nz, ny, nx).  Returns (y, cache)."""
    cache = []
    h = x
    for li, (W, b) in enumerate(params):
        z = conv3d(h, W, b, periodic)
        cache.append((h, z))
        h = gelu(z) if li < 3 else z
    return h, cache


def backward(params, cache, dy, periodic=True):
    """Gradients (dW, db) of every layer for the output gradient dy."""
    grads = [None] * 4
    g = dy
    for li in range(3, -1, -1):
        W, _ = params[li]
        h_in, z = cache[li]
        if li < 3:
            g = g * gelu_grad(z)
        grads[li] = conv3d_weight_grad(h_in, g, periodic)
        if li > 0:
            g = conv3d_input_grad(g, W, periodic)
    return grads


def rel_mse(y, t, mask=None):
    """Loss ||y - t||^2 / ||t||^2 over the masked points and its gradient dL/dy."""
    if mask is None:
        mask = np.ones_like(t, dtype=bool)
    d = np.where(mask, y - t, 0.0)
    tt = float(np.sum(np.where(mask, t, 0.0) ** 2))
    return float(np.sum(d * d)) / tt, 2.0 * d / tt


def adam_step(w, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of parameters w with gradient g at step t >= 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def flatten(params):
    """Flat parameter vector in the library's order: per layer W (Cout, Cin, 3, 3, 3) then b."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(flat):
    params, o = [], 0
    for li in range(4):
        ci, co = CHANNELS[li], CHANNELS[li + 1]
        nw = co * ci * 27
        W = flat[o:o + nw].reshape(co, ci, 3, 3, 3)
        o += nw
        b = flat[o:o + co]
        o += co
        params.append((W, b))
    return params


def num_params():
    return sum(CHANNELS[i + 1] * CHANNELS[i] * 27 + CHANNELS[i + 1] for i in range(4))


# ---- operator-weighted loss: the residual left after the learned stage ------------------
_NBR = {0: (0, 0, 1), 1: (0, 0, -1), 2: (0, 1, 0), 3: (0, -1, 0), 4: (1, 0, 0), 5: (-1, 0, 0)}  # (dk, dj, di) of E,W,N,S,U,D


def _shift(f, dk, dj, di, seg):
    """g[p] = f[p + (dk, dj, di)] on (nz, ny, nx) with zero outside the field and outside p's own
    segment of seg rows in j (stacked crops); no wrap."""
    nz, ny, nx = f.shape
    g = np.zeros_like(f)
    ks, ke = max(0, -dk), nz - max(0, dk)
    is_, ie = max(0, -di), nx - max(0, di)
    for s0 in range(0, ny, seg):
        js, je = s0 + max(0, -dj), s0 + seg - max(0, dj)
        g[ks:ke, js:je, is_:ie] = f[ks + dk:ke + dk, js + dj:je + dj, is_ + di:ie + di]
    return g


def ahat_crop(bands, d, seg=None):
    """(Ahat d)[p] = d[p] + sum_b band_b[p] d[p + offset_b] on a training crop (nz, ny, nx) whose
    neighbours outside the crop (or its segment of seg rows) are absent; bands (6, nz, ny, nx)."""
    seg = seg or d.shape[1]
    out = d.copy()
    for b, (dk, dj, di) in _NBR.items():
        out += bands[b] * _shift(d, dk, dj, di, seg)
    return out


def ahat_crop_transpose(bands, w, seg=None):
    """The adjoint of ahat_crop: (Ahat^T w)[q] = w[q] + sum_b band_b[q - offset_b] w[q - offset_b]."""
    seg = seg or w.shape[1]
    out = w.copy()
    for b, (dk, dj, di) in _NBR.items():
        out += _shift(bands[b] * w, -dk, -dj, -di, seg)
    return out


def op_loss(y, t, bands, mask, seg=None):
    """Loss ||mask Ahat (y - t)||^2 / ||mask Ahat t||^2 and its gradient dL/dy
    = 2 Ahat^T (mask Ahat (y - t)) / ||mask Ahat t||^2.  With t = Ahat^-1 e1 (the stage's target),
    Ahat t = e1 and the loss is the squared relative residual left after the stage."""
    u = np.where(mask, ahat_crop(bands, y - t, seg), 0.0)
    at = np.where(mask, ahat_crop(bands, t, seg), 0.0)
    den = float(np.sum(at * at))
    return float(np.sum(u * u)) / den, 2.0 * ahat_crop_transpose(bands, u, seg) / den
