"""Failure detection without a GPU fault.

* the bounded device waits: a self-check kernel waits on an mbarrier on which
  nothing ever arrives; the wait gives up, OVS_ETIMEOUT is reported, and the
  context stays usable;
* a right-hand side with a NaN source is reported as OVS_EINVAL while the
  other right-hand sides of the same call are unaffected;
* a workspace request larger than the device gives OVS_ENOMEM, and the
  handle works afterwards.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import arnoldi, lattice

pytestmark = pytest.mark.gpu

MW = -1.5
DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _small(gpu, mu=0.3):
    dims = (4, 4, 4, 4)
    links = synth.gauge_links(dims, 1, 0.5)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, mu, MW)
    return g, lattice.hw_operator(links, dims, mu, MW)


def test_bounded_wait_reports_timeout_and_context_survives(gpu):
    assert gpu.check_wait_timeout() == -7  # OVS_ETIMEOUT
    g, h = _small(gpu)
    x = synth.gaussian_vectors(3072, 2, 3)
    xd = torch.from_numpy(x).to(DEV)
    yd = torch.empty_like(xd)
    gpu.matvec(g, 1, xd, yd, prec=gpu.F64)
    assert rel(yd.cpu().numpy()[1], h @ x[1]) < 1e-13
    g.destroy()


def test_nonfinite_source_is_flagged_per_rhs(gpu):
    g, h = _small(gpu)
    x = synth.gaussian_vectors(3072, 3, 4)
    x[1, 17] = np.nan
    xd = torch.from_numpy(x).to(DEV)
    yd = torch.empty_like(xd)
    gpu.sign_apply(g, xd, yd, 40, prec=gpu.F64, want_info=False)
    with pytest.raises(gpu.OvsError, match="EINVAL.*right-hand side 1"):
        gpu.get_info(g, 3)
    y = yd.cpu().numpy()
    for r in (0, 2):
        ref, _ = arnoldi.arnoldi_sign(lambda q: h @ q, x[r], 40)
        assert rel(y[r], ref) < 1e-12
    g.destroy()


def test_workspace_too_large_gives_enomem_then_recovers(gpu):
    dims = (16, 16, 16, 16)  # N = 786,432
    g = gpu.create_gauge(dims, 1, 0.5, gpu.MIXED)
    gpu.set_mu(g, 0.2, MW)
    n = 12 * int(np.prod(dims))
    free, total = torch.cuda.mem_get_info()
    nrhs = 64  # basis 64 x 791 x N x 8 B = 318 GB, beyond the device
    assert nrhs * 791 * n * 8 > total
    x = torch.zeros((nrhs, n), dtype=torch.complex128, device=DEV)
    x[:, 0] = 1.0
    y = torch.empty_like(x)
    with pytest.raises(gpu.OvsError, match="ENOMEM"):
        gpu.sign_apply(g, x, y, 790, prec=gpu.MIXED)
    del x, y
    # the handle still works at a size that fits
    x1 = torch.from_numpy(synth.gaussian_vectors(n, 1, 6)).to(DEV)
    y1 = torch.empty_like(x1)
    st, info = gpu.sign_apply(g, x1, y1, 20, prec=gpu.MIXED)
    assert st == 0 and info[0]["k_used"] == 20
    assert torch.isfinite(y1).all()
    g.destroy()
