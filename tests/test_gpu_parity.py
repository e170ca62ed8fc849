"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Tolerances (relative 2-norm per right-hand side):
* FP64 matvec vs the sparse oracle operator: 1e-13;
* mixed (complex64) matvec: 2e-6 (float rounding of links and spinors);
* FP64 sign application vs the oracle's CGS2 Arnoldi at equal (m, k): 1e-12;
* mixed sign application vs the FP64 oracle at equal (m, k): 1e-6.
"""

import numpy as np
import pytest
import torch

import synth
from oracle import arnoldi, deflation, freefield, lattice, signfun

pytestmark = pytest.mark.gpu

MU, MW = 0.3, -1.5
DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


@pytest.fixture(scope="module")
def small(gpu):
    """4^4 lattice, eps 0.5, seed 1 (the tiny configuration)."""
    dims = (4, 4, 4, 4)
    links = synth.gauge_links(dims, 1, 0.5)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, MU, MW)
    h = lattice.hw_operator(links, dims, MU, MW)
    return g, h, dims


# ------------------------------------------------------------------ links
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 2, 5, 4)])
def test_create_gauge_matches_generator(gpu, dims):
    g = gpu.create_gauge(dims, 3, 0.7, gpu.F64)
    got = gpu.get_links(g)
    ref = synth.gauge_links(dims, 3, 0.7)
    assert np.abs(got - ref).max() < 1e-13
    g.destroy()


def test_links_roundtrip(gpu):
    dims = (2, 3, 2, 4)
    links = synth.gauge_links(dims, 5, 0.6) * 1.5  # not unitary on purpose
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    assert np.array_equal(gpu.get_links(g), links)
    g.destroy()


# ----------------------------------------------------------------- matvec
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 8), (3, 4, 5, 6), (8, 8, 8, 8)])
@pytest.mark.parametrize("nrhs", [1, 3])
@pytest.mark.parametrize("op", [0, 1, 2])
def test_matvec_f64_and_mixed(gpu, dims, nrhs, op):
    v = int(np.prod(dims))
    links = synth.gauge_links(dims, 7, 0.6)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, MU, MW)
    x = synth.gaussian_vectors(12 * v, nrhs, 4)
    d = lattice.wilson_dirac(links, dims, MU, MW)
    h = lattice.hw_operator(links, dims, MU, MW)
    ref_op = {0: lambda z: d @ z, 1: lambda z: h @ z, 2: lambda z: h @ (h @ z)}[op]
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    for prec, tol in ((gpu.F64, 1e-13), (gpu.MIXED, 2e-6)):
        gpu.matvec(g, op, xd, yd, prec=prec)
        y = yd.cpu().numpy()
        for r in range(nrhs):
            assert rel(y[r], ref_op(x[r])) < tol, (prec, r)
    g.destroy()


def test_matvec_sixteen_rhs_and_host_buffers(gpu):
    dims = (4, 4, 4, 4)
    links = synth.gauge_links(dims, 2, 0.5)
    g = gpu.create_gauge_from_links(dims, links, gpu.F64)
    gpu.set_mu(g, 0.1, MW)
    h = lattice.hw_operator(links, dims, 0.1, MW)
    x = synth.gaussian_vectors(3072, 16, 9)
    y = np.empty_like(x)
    gpu.matvec(g, 1, x, y, prec=gpu.F64)  # host numpy buffers
    for r in (0, 7, 15):
        assert rel(y[r], h @ x[r]) < 1e-13
    g.destroy()


def test_matvec_free_field_closed_form(gpu):
    dims = (8, 4, 6, 10)
    v = int(np.prod(dims))
    g = gpu.create_gauge_from_links(dims, synth.unit_links(dims), gpu.F64)
    gpu.set_mu(g, 0.25, -1.2)
    x = synth.gaussian_vectors(12 * v, 1, 3)
    yd = torch.empty((1, 12 * v), dtype=torch.complex128, device=DEV)
    gpu.matvec(g, 1, to_dev(x), yd, prec=gpu.F64)
    ref = freefield.apply_free(x[0], dims, 0.25, -1.2, "H")
    assert rel(yd.cpu().numpy()[0], ref) < 1e-13
    g.destroy()


# ------------------------------------------------------------ sign apply
@pytest.mark.parametrize("nrhs,k", [(1, 30), (3, 41)])
def test_sign_apply_f64_undeflated_matches_cpu_arnoldi(gpu, small, nrhs, k):
    g, h, dims = small
    x = synth.gaussian_vectors(3072, nrhs, 2)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    st, info = gpu.sign_apply(g, xd, yd, k, prec=gpu.F64)
    assert st == 0
    y = yd.cpu().numpy()
    for r in range(nrhs):
        ref, oinfo = arnoldi.arnoldi_sign(lambda q: h @ q, x[r], k)
        assert info[r]["k_used"] == oinfo["k_used"] == k
        assert info[r]["beta"] == pytest.approx(oinfo["beta"], rel=1e-14)
        assert rel(y[r], ref) < 1e-12


def test_sign_apply_mixed_undeflated(gpu, small):
    g, h, dims = small
    x = synth.gaussian_vectors(3072, 2, 5)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    gpu.sign_apply(g, xd, yd, 40, prec=gpu.MIXED)
    y = yd.cpu().numpy()
    for r in range(2):
        ref, _ = arnoldi.arnoldi_sign(lambda q: h @ q, x[r], 40)
        assert rel(y[r], ref) < 1e-6


def test_sign_apply_ones_source(gpu, small):
    """The paper's source x = (1, ..., 1) (Fig. DeflArn)."""
    g, h, dims = small
    x = synth.ones_vector(3072)
    yd = torch.empty((1, 3072), dtype=torch.complex128, device=DEV)
    gpu.sign_apply(g, to_dev(x), yd, 20, prec=gpu.F64)
    ref, _ = arnoldi.arnoldi_sign(lambda q: h @ q, x[0], 20)
    assert rel(yd.cpu().numpy()[0], ref) < 1e-12


@pytest.fixture(scope="module")
def deflated_problem(gpu):
    """2x4x4x4 lattice (N = 1536) with exact critical eigenpairs (dense)."""
    dims = (2, 4, 4, 4)
    links = synth.gauge_links(dims, 4, 0.7)
    h = lattice.hw_operator(links, dims, 0.2, MW)
    hd = h.toarray()
    dec = signfun.eig_decomposition(hd)
    lam, R, L = deflation.critical_pairs_dense(hd, 16, dec)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, 0.2, MW)
    gpu.deflate_load(g, R.T.copy(), L.T.copy(), lam)
    return g, h, hd, dec, lam, R, L


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6)])
def test_sign_apply_deflated_matches_cpu(gpu, deflated_problem, prec, tol):
    g, h, hd, dec, lam, R, L = deflated_problem
    x = synth.gaussian_vectors(1536, 3, 8)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    gpu.sign_apply(g, xd, yd, 36, prec=prec)
    y = yd.cpu().numpy()
    for r in range(3):
        ref, oinfo = deflation.lr_sign_apply(lambda q: h @ q, x[r], R, L, lam, 36)
        assert rel(y[r], ref) < tol
    # and deflation helps against the exact sign
    exact = signfun.sgn_apply_dense(hd, x[0], dec)
    y_undefl, _ = arnoldi.arnoldi_sign(lambda q: h @ q, x[0], 36)
    assert rel(y[0], exact) < rel(y_undefl, exact)


def test_deflated_large_k_reaches_exact(gpu, deflated_problem):
    """With m = 16 and k = 400 the method is within 1e-10 of the dense sgn."""
    g, h, hd, dec, lam, R, L = deflated_problem
    x = synth.gaussian_vectors(1536, 1, 3)
    yd = torch.empty((1, 1536), dtype=torch.complex128, device=DEV)
    gpu.sign_apply(g, to_dev(x), yd, 400, prec=gpu.F64)
    exact = signfun.sgn_apply_dense(hd, x[0], dec)
    ref, _ = deflation.lr_sign_apply(lambda q: h @ q, x[0], R, L, lam, 400)
    assert rel(ref, exact) < 1e-10
    assert rel(yd.cpu().numpy()[0], exact) < 1e-10


def test_source_in_deflated_space(gpu, deflated_problem):
    """x in span(R): x_ominus = 0, beta = 0, y = R sgn(Lambda) L^+ x exactly."""
    g, h, hd, dec, lam, R, L = deflated_problem
    x = (R[:, 2] + 0.5j * R[:, 7])[None, :]
    yd = torch.empty((1, 1536), dtype=torch.complex128, device=DEV)
    st, info = gpu.sign_apply(g, to_dev(x), yd, 20, prec=gpu.F64)
    assert info[0]["beta"] < 1e-12
    ref = np.sign(lam[2].real) * R[:, 2] + 0.5j * np.sign(lam[7].real) * R[:, 7]
    assert rel(yd.cpu().numpy()[0], ref) < 1e-10


def test_zero_source(gpu, small):
    g, h, dims = small
    xd = torch.zeros((2, 3072), dtype=torch.complex128, device=DEV)
    yd = torch.full_like(xd, 7.0)
    st, info = gpu.sign_apply(g, xd, yd, 10, prec=gpu.MIXED)
    assert torch.count_nonzero(yd).item() == 0
    assert info[0]["k_used"] == 0 and info[0]["beta"] == 0.0


def test_breakdown_free_field_exact(gpu):
    """Plane-wave source on the free field: the Krylov space is invariant
    after <= 4 steps; the result equals the closed form sgn(H)x."""
    dims = (8, 8, 8, 16)
    v = int(np.prod(dims))
    g = gpu.create_gauge_from_links(dims, synth.unit_links(dims), gpu.MIXED)
    gpu.set_mu(g, MU, MW)
    x = synth.plane_wave_vectors(dims, [(1, 0, 0, 0), (0, 2, 1, 3)], 7)
    yd = torch.empty((1, 12 * v), dtype=torch.complex128, device=DEV)
    st, info = gpu.sign_apply(g, to_dev(x), yd, 30, prec=gpu.F64)
    assert info[0]["k_used"] <= 4
    ref = freefield.apply_free(x[0], dims, MU, MW, "sgnH")
    assert rel(yd.cpu().numpy()[0], ref) < 1e-12


def test_breakdown_pure_gauge_exact(gpu):
    """Gauge covariance: the same on a pure-gauge field (non-trivial links)."""
    dims = (4, 4, 4, 8)
    v = int(np.prod(dims))
    u, om = synth.pure_gauge_links(dims, 11)
    g = gpu.create_gauge_from_links(dims, u, gpu.MIXED)
    gpu.set_mu(g, MU, MW)
    x = synth.plane_wave_vectors(dims, [(1, 1, 0, 2)], 2, omega=om)
    yd = torch.empty((1, 12 * v), dtype=torch.complex128, device=DEV)
    for prec, tol in ((gpu.F64, 1e-12), (gpu.MIXED, 1e-6)):
        st, info = gpu.sign_apply(g, to_dev(x), yd, 30, prec=prec)
        ref = freefield.apply_free(x[0], dims, MU, MW, "sgnH", omega=om)
        assert rel(yd.cpu().numpy()[0], ref) < tol


def test_host_buffers_sign_apply(gpu, small):
    g, h, dims = small
    x = synth.gaussian_vectors(3072, 2, 6)
    y_host = np.empty_like(x)
    gpu.sign_apply(g, x, y_host, 24, prec=gpu.F64)
    yd = torch.empty((2, 3072), dtype=torch.complex128, device=DEV)
    gpu.sign_apply(g, to_dev(x), yd, 24, prec=gpu.F64)
    assert np.array_equal(y_host, yd.cpu().numpy())


def test_deflation_save_restore(gpu, deflated_problem, tmp_path):
    g, h, hd, dec, lam, R, L = deflated_problem
    path = str(tmp_path / "defl.bin")
    gpu.deflate_save(g, path)
    R1, L1, lam1 = gpu.deflate_get(g)
    gpu.deflate_restore(g, path)
    R2, L2, lam2 = gpu.deflate_get(g)
    assert np.allclose(R1, R2, atol=1e-15) and np.allclose(L1, L2, atol=1e-14)
    assert np.array_equal(lam1, lam2)
    # biorthonormal after installation
    G = L2.conj() @ R2.T
    assert np.abs(G - np.eye(len(lam2))).max() < 1e-12


def test_errors(gpu):
    dims = (2, 2, 2, 2)
    g = gpu.create_gauge(dims, 1, 0.5, gpu.F64)
    x = torch.zeros((1, 192), dtype=torch.complex128, device=DEV)
    with pytest.raises(gpu.OvsError, match="ESTATE"):
        gpu.sign_apply(g, x, x.clone(), 4, prec=gpu.F64)
    gpu.set_mu(g, 0.1, MW)
    with pytest.raises(gpu.OvsError, match="ESTATE"):  # handle without complex64 copies
        gpu.sign_apply(g, x, x.clone(), 4, prec=gpu.MIXED)
    with pytest.raises(gpu.OvsError, match="EINVAL"):
        gpu.sign_apply(g, x, x.clone(), 0, prec=gpu.F64)
    lam = np.array([0.0 + 1j])
    with pytest.raises(gpu.OvsError, match="ESIGN"):
        gpu.deflate_load(g, np.ones((1, 192)), np.ones((1, 192)), lam)
    g.destroy()
