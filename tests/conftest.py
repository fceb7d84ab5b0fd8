import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libhz.so")
    config.addinivalue_line("markers", "slow: long-running")


def pytest_collection_modifyitems(config, items):
    try:
        import torch

        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def dense_operator(A):
    """Assemble the 7-band operator as a dense matrix (independent index code for pins).

    Row p = (k, j, i); band b couples p to its neighbour; i wraps, j and k do not.
    """
    _, nz, ny, nx = A.shape
    n = nx * ny * nz
    M = np.zeros((n, n))
    offs = {1: (1, 0, 0), 2: (-1, 0, 0), 3: (0, 1, 0), 4: (0, -1, 0), 5: (0, 0, 1), 6: (0, 0, -1)}
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                row = (k * ny + j) * nx + i
                M[row, row] += A[0, k, j, i]
                for b, (di, dj, dk) in offs.items():
                    ii, jj, kk = (i + di) % nx, j + dj, k + dk
                    if 0 <= jj < ny and 0 <= kk < nz:
                        M[row, (kk * ny + jj) * nx + ii] += A[b, k, j, i]
                    else:
                        assert A[b, k, j, i] == 0.0
    return M


def dense_from_hat(Ah):
    """Dense matrix of Ahat = I + off-diagonal bands."""
    _, nz, ny, nx = Ah.shape
    A7 = np.concatenate([np.ones((1, nz, ny, nx)), Ah], axis=0)
    return dense_operator(A7)
