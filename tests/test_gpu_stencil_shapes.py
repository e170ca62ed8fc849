"""Stencil launch shapes and their autotuner.

Every shape (1 or 2 right-hand sides per thread; blocks of 32, 64 or 128
sites times 1 to 8 right-hand-side tiles, at most 256 threads) must give
bit-identical results that match the oracle operator;
the autotuner must time every candidate and keep the fastest; pinned shapes
with multi-RHS tiles must leave a convergence-stopped application (where
some right-hand sides of a tile stop early) unchanged to the bit.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import lattice

pytestmark = pytest.mark.gpu

MW = -1.5
DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_every_shape_bit_identical_and_correct(gpu):
    dims, mu, nrhs = (8, 4, 6, 10), 0.2, 7  # V = 1920: ragged for 256-site blocks; 7 RHS: ragged tiles
    v = int(np.prod(dims))
    links = synth.gauge_links(dims, 9, 0.6)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, mu, MW)
    h = lattice.hw_operator(links, dims, mu, MW)
    x = synth.gaussian_vectors(12 * v, nrhs, 31)
    xd = torch.from_numpy(x).to(DEV)
    yd = torch.empty_like(xd)
    for prec, tol in ((gpu.F64, 1e-13), (gpu.MIXED, 2e-6)):
        outs = []
        for shape in gpu.STENCIL_SHAPES:
            gpu.set_stencil_shape(g, prec, nrhs, shape)
            gpu.matvec(g, 1, xd, yd, prec=prec)
            assert gpu.stencil_tuning(g, prec, nrhs)["shape"] == shape
            outs.append(yd.clone())
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        y = outs[0].cpu().numpy()
        for r in range(nrhs):
            assert rel(y[r], h @ x[r]) < tol
        gpu.set_stencil_shape(g, prec, nrhs, None)  # forget: the next launch tunes
        assert gpu.stencil_tuning(g, prec, nrhs) is None
        gpu.matvec(g, 1, xd, yd, prec=prec)
        info = gpu.stencil_tuning(g, prec, nrhs)
        timed = {sh: t for sh, t in info["ms"].items() if t > 0}
        expect = [sh for sh in gpu.STENCIL_SHAPES if prec == gpu.MIXED or sh[0] == 1]
        assert sorted(timed) == sorted(expect)
        assert timed[info["shape"]] == min(timed.values())
        assert torch.equal(yd, outs[0])
    with pytest.raises(gpu.OvsError, match="EINVAL"):
        gpu.set_stencil_shape(g, gpu.F64, nrhs, (3, 128, 1))
    g.destroy()


def test_pinned_tile_with_early_stops_is_bit_identical(gpu):
    dims, mu, nrhs = (4, 4, 4, 4), 0.3, 6
    links = synth.gauge_links(dims, 1, 0.5)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, mu, MW)
    x = synth.gaussian_vectors(3072, nrhs, 22)
    x[1] *= 0.0  # stops at once
    x[2] = synth.ones_vector(3072)[0]
    xd = torch.from_numpy(x).to(DEV)
    results = []
    for shape in ((1, 128, 1), (2, 32, 4), (1, 32, 8), (2, 128, 2)):
        gpu.set_stencil_shape(g, gpu.MIXED, nrhs, shape)
        yd = torch.empty_like(xd)
        st, info = gpu.sign_apply(g, xd, yd, 200, prec=gpu.MIXED, check_every=10, tol=1e-5)
        results.append((yd, [(i["k_used"], i["status"]) for i in info]))
    ks = [k for k, _ in results[0][1]]
    assert len(set(ks)) > 1  # the right-hand sides of a tile stop at different steps
    for yd, info in results[1:]:
        assert info == results[0][1]
        assert torch.equal(yd, results[0][0])
    g.destroy()
