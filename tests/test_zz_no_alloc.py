"""hz_dot_noalloc against hz_dot and the CPU oracle's dot product (GPU).

hz_dot_noalloc exists for callers that cannot allocate device memory (a fixed
memory pool, an allocator owned by another framework, a no-allocation rule
after start-up): it keeps its scratch in a static device array instead of
memory from cudaMalloc.  Its result must equal hz_dot's, and the oracle's
FP64 dot product of the same values, within the dot tolerance of the other
tests, on two calls in a row (the second call starts from the scratch the
first one left behind).  This file is collected last.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [1, 1000, 138240, 3 << 20])
def test_dot_noalloc_matches_hz_dot_twice(prec, n):
    import torch

    import paper_1811_03852_gb300 as hz

    dt = torch.float64 if prec == "fp64" else torch.float32
    x = torch.from_numpy(gen.normals(41, 0, n)).to(dt).cuda()
    y = torch.from_numpy(gen.normals(42, 0, n)).to(dt).cuda()
    ref = hz.dot(x, y)
    xh, yh = x.double().cpu().numpy(), y.double().cpu().numpy()
    ref_oracle = oracle.dot(xh, yh)
    scale = float(np.dot(np.abs(xh), np.abs(yh)))
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    vals = []
    for _ in range(2):
        out.fill_(np.nan)
        hz.dot_noalloc(x, y, out)
        torch.cuda.synchronize()
        vals.append(float(out.item()))
    for v in vals:
        assert abs(v - ref) <= 1e-13 * scale, (v, ref)
        assert abs(v - ref_oracle) <= 1e-13 * scale, (v, ref_oracle)
    assert vals[0] == vals[1]


def test_dot_noalloc_rejects_bad_arguments():
    import ctypes

    import paper_1811_03852_gb300 as hz

    L = hz.load()
    assert L.hz_dot_noalloc(hz.HZ_PREC_FP32, -1, None, None, None, ctypes.c_void_p(8)) == hz.HZ_ERR_INVALID
    assert L.hz_dot_noalloc(7, 4, ctypes.c_void_p(8), ctypes.c_void_p(8), None, ctypes.c_void_p(8)) == hz.HZ_ERR_INVALID
