"""Helpers shared by the GPU tests (inputs from gen/, references from oracle/)."""
import numpy as np


def dev(a, dtype=None):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    import torch

    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def abs_matvec_hat(Ah, x):
    """(|Ahat| |x|) elementwise: the scale of the rounding error of Ahat x."""
    import oracle

    return oracle.matvec_hat(np.abs(Ah), np.abs(x))
