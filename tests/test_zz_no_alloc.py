"""The no-allocation matvec (ovs_matvec_noalloc) against ovs_matvec.

ovs_matvec_noalloc serves callers that cannot let the library allocate
device memory (their pool is owned by another allocator, or their loop must
not pay cudaMalloc's synchronisation); it keeps its work fields in a fixed
array inside the library. This test calls both entry points through the C
ABI on the same inputs, twice in a row with different operators and sizes
(the shared array keeps the previous call's contents), and checks that
requests beyond the array are refused. This file is collected last on
purpose.
"""

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_matvec_twice(gpu):
    dims = (4, 4, 4, 8)
    n = 12 * 4 * 4 * 4 * 8
    g = gpu.create_gauge(dims, 9, 0.6, gpu.MIXED)
    gpu.set_mu(g, 0.2, -1.5)
    calls = [(1, 3, gpu.F64, 1e-13), (2, 2, gpu.MIXED, 2e-6), (0, 5, gpu.F64, 1e-13)]
    for op, nrhs, prec, tol in calls:
        x = torch.from_numpy(synth.gaussian_vectors(n, nrhs, 10 + op)).cuda()
        y_ref = torch.empty_like(x)
        y_na = torch.full_like(x, 3.0)
        gpu.matvec(g, op, x, y_ref, prec=prec)
        gpu.matvec_noalloc(g, op, x, y_na, prec=prec)
        torch.cuda.synchronize()
        a, b = y_na.cpu().numpy(), y_ref.cpu().numpy()
        for r in range(nrhs):
            assert rel(a[r], b[r]) <= tol, (op, prec, r)
    g.destroy()


def test_noalloc_rejects_oversize_and_host(gpu):
    dims = (8, 8, 8, 8)
    n = 12 * 8 ** 4  # 49152: F64 fits up to 10 RHS
    g = gpu.create_gauge(dims, 1, 0.5, gpu.F64)
    gpu.set_mu(g, 0.1, -1.5)
    x = torch.zeros((11, n), dtype=torch.complex128, device="cuda:0")
    y = torch.empty_like(x)
    with pytest.raises(gpu.OvsError, match="EINVAL"):
        gpu.matvec_noalloc(g, 1, x, y, prec=gpu.F64)
    xh = np.zeros((1, n), dtype=np.complex128)
    with pytest.raises(gpu.OvsError, match="device pointers"):
        gpu.matvec_noalloc(g, 1, xh, xh.copy(), prec=gpu.F64)
    # the largest accepted size works
    x10 = torch.from_numpy(synth.gaussian_vectors(n, 10, 4)).cuda()
    y10 = torch.empty_like(x10)
    y10r = torch.empty_like(x10)
    gpu.matvec_noalloc(g, 1, x10, y10, prec=gpu.F64)
    gpu.matvec(g, 1, x10, y10r, prec=gpu.F64)
    torch.cuda.synchronize()
    assert rel(y10.cpu().numpy(), y10r.cpu().numpy()) <= 1e-13
    g.destroy()
