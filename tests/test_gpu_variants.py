"""GPU parity of the method's variants through the C ABI: Schur deflation
with the App. A Sylvester solver (Sec. 5.2), the harmonic variant (Sec. 4),
the overlap operator D_ov (Sec. 2, Eqs. Dov, GW:eq) with its nested
inversion, and the orthogonality and Arnoldi relation of the device basis.

Tolerances (relative 2-norm per right-hand side):
* FP64 vs the oracle at equal (m, k): 1e-12 (Schur: 1e-11, the App. A
  recurrences amplify rounding of the first column of Y by up to ~1e2 at
  k ~ 60 here);
* mixed vs the FP64 oracle at equal (m, k): 1e-6;
* Ginsparg-Wilson relation and the overlap solve: bounds derived from the
  inner sign's measured error against the dense sign.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import synth
from oracle import arnoldi, deflation, lattice, overlap, schur, signfun

pytestmark = pytest.mark.gpu

MW = -1.5
DEV = "cuda:0"


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def g5(x):
    return x * lattice.gamma5_diag(x.shape[-1] // 12)


@pytest.fixture(scope="module")
def tiny(gpu):
    """2x2x2x4 lattice (N = 384), mu = 0.3: the dense sign is cheap."""
    dims, mu = (2, 2, 2, 4), 0.3
    links = synth.gauge_links(dims, 1, 0.5)
    h = lattice.hw_operator(links, dims, mu, MW)
    hd = h.toarray()
    dec = np.linalg.eig(hd)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, mu, MW)
    yield g, h, hd, dec
    g.destroy()


@pytest.fixture(scope="module")
def small(gpu):
    """4^4 lattice, eps 0.5, seed 1, mu 0.3 (the tiny configuration)."""
    dims, mu = (4, 4, 4, 4), 0.3
    links = synth.gauge_links(dims, 1, 0.5)
    h = lattice.hw_operator(links, dims, mu, MW)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, mu, MW)
    yield g, h, links, dims, mu
    g.destroy()


# ---------------------------------------------------------- harmonic (Sec. 4)
@pytest.mark.parametrize("k", [31, 40])
def test_harmonic_matches_oracle(gpu, small, k):
    g, h, links, dims, mu = small
    gpu.deflate_load(g, np.zeros((0, 3072)), np.zeros((0, 3072)), np.zeros(0))
    x = synth.gaussian_vectors(3072, 2, 12)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    for prec, tol in ((gpu.F64, 1e-12), (gpu.MIXED, 1e-6)):
        st, info = gpu.sign_apply(g, xd, yd, k, prec=prec, harmonic=True)
        assert st == 0
        y = yd.cpu().numpy()
        for r in range(2):
            ref, _ = arnoldi.arnoldi_sign(lambda q: h @ q, x[r], k, harmonic=True)
            assert rel(y[r], ref) < tol, (prec, r)


def test_harmonic_lr_deflated_matches_oracle(gpu, small):
    g, h, links, dims, mu = small
    R, L, lam = synth.synthetic_deflation(3072, 12, 501)
    gpu.deflate_load(g, R.T.copy(), L.T.copy(), lam)
    x = synth.gaussian_vectors(3072, 3, 13)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    gpu.sign_apply(g, xd, yd, 37, prec=gpu.F64, harmonic=True)
    y = yd.cpu().numpy()
    for r in range(3):
        ref, _ = deflation.lr_sign_apply(lambda q: h @ q, x[r], R, L, lam, 37, harmonic=True)
        assert rel(y[r], ref) < 1e-12
    gpu.deflate_load(g, np.zeros((0, 3072)), np.zeros((0, 3072)), np.zeros(0))


def test_harmonic_removes_see_saw_on_gpu(gpu, tiny):
    """Sec. 4: plain Arnoldi alternates between odd and even k, the harmonic
    form decreases smoothly (errors against the dense sign)."""
    g, h, hd, dec = tiny
    x = synth.gaussian_vectors(384, 1, 2)
    ref = signfun.sgn_apply_dense(hd, x[0], dec)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    plain, harm = [], []
    for k in range(30, 38):
        gpu.sign_apply(g, xd, yd, k, prec=gpu.F64)
        plain.append(rel(yd.cpu().numpy()[0], ref))
        gpu.sign_apply(g, xd, yd, k, prec=gpu.F64, harmonic=True)
        harm.append(rel(yd.cpu().numpy()[0], ref))
    assert min(plain[i + 1] / plain[i] for i in range(0, 7, 2)) > 1.5
    assert all(harm[i + 1] <= harm[i] * 1.01 for i in range(7))


def test_harmonic_flag_errors(gpu, small):
    g, h, links, dims, mu = small
    xd = torch.zeros((1, 3072), dtype=torch.complex128, device=DEV)
    with pytest.raises(gpu.OvsError, match="EINVAL"):
        gpu.sign_apply(g, xd, xd.clone(), 20, prec=gpu.F64, harmonic=True, check_every=10, tol=1e-6)


# ------------------------------------------------------- overlap (Sec. 2)
def test_overlap_apply_matches_oracle(gpu, small):
    g, h, links, dims, mu = small
    R, L, lam = synth.synthetic_deflation(3072, 10, 601)
    gpu.deflate_load(g, R.T.copy(), L.T.copy(), lam)
    x = synth.gaussian_vectors(3072, 2, 14)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    for prec, tol in ((gpu.F64, 1e-12), (gpu.MIXED, 1e-6)):
        gpu.overlap_apply(g, xd, yd, 30, prec=prec)
        y = yd.cpu().numpy()
        for r in range(2):
            ref = overlap.dov_apply(lambda q: deflation.lr_sign_apply(lambda z: h @ z, q, R, L, lam, 30)[0], x[r])
            assert rel(y[r], ref) < tol, (prec, r)
    # host buffers give the same bits
    yh = np.empty_like(x)
    gpu.overlap_apply(g, x, yh, 30, prec=gpu.F64)
    gpu.overlap_apply(g, xd, yd, 30, prec=gpu.F64)
    assert np.array_equal(yh, yd.cpu().numpy())
    gpu.deflate_load(g, np.zeros((0, 3072)), np.zeros((0, 3072)), np.zeros(0))


def _exact_lr(hd, dec, m):
    lam, R, L = deflation.critical_pairs_dense(hd, m, dec)
    return lam, R, L


def test_ginsparg_wilson_on_gpu(gpu, tiny):
    """{D_ov, gamma5} x = D_ov gamma5 D_ov x (Eq. GW:eq) with the GPU D_ov,
    to the accuracy of its sign (measured against the dense sign)."""
    g, h, hd, dec = tiny
    lam, R, L = _exact_lr(hd, dec, 60)
    gpu.deflate_load(g, R.T.copy(), L.T.copy(), lam)
    x = synth.gaussian_vectors(384, 2, 21)
    k = 200
    dov = lambda v: (lambda vd, yd: (gpu.overlap_apply(g, vd, yd, k, prec=gpu.F64), yd.cpu().numpy())[1])(
        to_dev(v), torch.empty((v.shape[0], 384), dtype=torch.complex128, device=DEV))
    d_x = dov(x)
    d_g5x = dov(g5(x))
    d_g5_d_x = dov(g5(d_x))
    sg = signfun.sgn_matrix(hd)
    err_sign = max(rel(d_x[r] - x[r], g5(sg @ x[r])) for r in range(2))
    assert err_sign < 1e-11
    for r in range(2):
        assert rel(d_g5x[r] + g5(d_x[r]), d_g5_d_x[r]) < 1e-10
    gpu.deflate_load(g, np.zeros((0, 384)), np.zeros((0, 384)), np.zeros(0))


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-5)])
def test_overlap_solve_matches_dense(gpu, tiny, prec, tol):
    """Nested inversion: GMRES(8) (several cycles) around D_ov against the
    dense solve of D_ov x = b, with an inner sign accurate to ~1e-12."""
    g, h, hd, dec = tiny
    lam, R, L = _exact_lr(hd, dec, 60)
    gpu.deflate_load(g, R.T.copy(), L.T.copy(), lam)
    b = synth.gaussian_vectors(384, 2, 31)
    x = np.empty_like(b)
    st, info = gpu.overlap_solve(g, b, x, 200, restart=8, tol=tol, max_cycles=60, prec=prec)
    assert st == 0, info
    dd = overlap.dov_dense(signfun.sgn_matrix(hd))
    for r in range(2):
        assert info[r]["rel_resid"] <= tol and info[r]["cycles"] > 1
        xr = np.linalg.solve(dd, b[r])
        assert rel(x[r], xr) < 50 * tol, r
    # the oracle's GMRES with the same reading takes the same number of steps
    _, oinfo = overlap.gmres(lambda q: dd @ q, b[0], 8, tol, 60)
    if prec == 0:
        assert abs(oinfo["iters"] - info[0]["iters"]) <= 2 * 8
    gpu.deflate_load(g, np.zeros((0, 384)), np.zeros((0, 384)), np.zeros(0))


def test_overlap_solve_reports_not_converged(gpu, tiny):
    g, h, hd, dec = tiny
    b = synth.gaussian_vectors(384, 1, 32)
    x = np.empty_like(b)
    st, info = gpu.overlap_solve(g, b, x, 40, restart=2, tol=1e-14, max_cycles=2, prec=gpu.F64)
    assert st == 1 and info[0]["status"] == 1 and info[0]["cycles"] == 2


# -------------------------------------------------------- Schur (Sec. 5.2)
def _schur_ref(h, S, T, x, k):
    return schur.schur_sign_apply(lambda q: h @ q, x, S, T, k)


@pytest.mark.parametrize("nrhs,k", [(1, 24), (3, 41)])
def test_schur_matches_oracle_tiny(gpu, tiny, nrhs, k):
    g, h, hd, dec = tiny
    lam_all, U = dec
    order = np.argsort(np.abs(lam_all.real), kind="stable")[:20]
    Rv = U[:, order]
    gpu.deflate_load_schur(g, Rv.T.copy())
    assert gpu.deflate_scheme(g) == "schur"
    S, T = schur.schur_from_eigvecs(lambda q: hd @ q, Rv)
    Sg, _, lam_g = gpu.deflate_get(g)
    assert np.abs(lam_g - np.diag(T)).max() < 1e-12
    assert np.abs(Sg.conj() @ Sg.T - np.eye(20)).max() < 1e-13
    x = synth.gaussian_vectors(384, nrhs, 41)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    for prec, tol in ((gpu.F64, 1e-11), (gpu.MIXED, 1e-6)):
        st, info = gpu.sign_apply(g, xd, yd, k, prec=prec)
        assert st == 0
        y = yd.cpu().numpy()
        for r in range(nrhs):
            ref, oinfo = _schur_ref(h, S, T, x[r], k)
            assert info[r]["k_used"] == oinfo["k_used"]
            assert rel(y[r], ref) < tol, (prec, r)
    gpu.deflate_load_schur(g, np.zeros((0, 384)))
    assert gpu.deflate_scheme(g) == "none"


def test_schur_full_krylov_exact_on_gpu(gpu, tiny):
    g, h, hd, dec = tiny
    lam_all, U = dec
    order = np.argsort(np.abs(lam_all.real), kind="stable")[:30]
    gpu.deflate_load_schur(g, U[:, order].T.copy())
    x = synth.gaussian_vectors(384, 1, 42)
    yd = torch.empty((1, 384), dtype=torch.complex128, device=DEV)
    gpu.sign_apply(g, to_dev(x), yd, 300, prec=gpu.F64)
    assert rel(yd.cpu().numpy()[0], signfun.sgn_apply_dense(hd, x[0], dec)) < 1e-10
    gpu.deflate_load_schur(g, np.zeros((0, 384)))


def test_schur_matches_oracle_8to4(gpu):
    """8^4 (N = 49,152), m = 30 seeded vectors as R (the construction and
    the formula are defined for any independent R), k = 60, 16 right-hand
    sides in one call: every right-hand side against the oracle. The seeded
    vectors are chirally projected, (1 +- gamma5) x / 2, so that the
    diagonal of T = S^H H_w S sits near +-1 (for H_w = gamma5 D_w and
    D_w = 1 - kappa (hops), s^H H_w s = +-s^H D_w s); plain Gaussian
    vectors give Rayleigh quotients near 0 and an ill-conditioned sgn(T)."""
    dims, mu = (8, 8, 8, 8), 0.2
    v = int(np.prod(dims))
    n, m, k, nrhs = 12 * v, 30, 60, 16
    links = synth.gauge_links(dims, 3, 0.7)
    h = lattice.hw_operator(links, dims, mu, MW)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, mu, MW)
    Rv = synth.gaussian_vectors(n, m, 701).T.copy()
    chi = lattice.gamma5_diag(v)[:, None] * np.where(np.arange(m) % 2 == 0, 1.0, -1.0)[None, :]
    Rv = 0.5 * (Rv + chi * Rv)
    gpu.deflate_load_schur(g, Rv.T.copy())
    S, T = schur.schur_from_eigvecs(lambda q: h @ q, Rv)
    x = synth.gaussian_vectors(n, nrhs, 702)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    st, _ = gpu.sign_apply(g, xd, yd, k, prec=gpu.F64)
    y64 = yd.cpu().numpy()
    st, _ = gpu.sign_apply(g, xd, yd, k, prec=gpu.MIXED)
    y32 = yd.cpu().numpy()
    for r in range(nrhs):
        ref, _ = _schur_ref(h, S, T, x[r], k)
        assert rel(y64[r], ref) < 1e-11, r
        assert rel(y32[r], ref) < 1e-6, r
    g.destroy()


def test_schur_device_setup(gpu):
    """ovs_deflate_setup_schur (right vectors only) at 6^4, m = 12, tol 1e-8: every
    eigenvalue on the diagonal of the installed T_m is one of the 2m
    eigenvalues of the sparse operator nearest 0 (ARPACK shift-invert), and
    the application
    with the installed S_m matches the oracle run on the same S_m."""
    dims, mu = (6, 6, 6, 6), 0.2
    v = int(np.prod(dims))
    links = synth.gauge_links(dims, 3, 0.6)
    h = lattice.hw_operator(links, dims, mu, MW)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, mu, MW)
    m = 12
    eig, st = gpu.deflate_setup(g, m, 1e-8, scheme="schur")
    assert st == 0 and gpu.deflate_scheme(g) == "schur"
    lam_ref = spla.eigs(h.tocsc(), k=2 * m, sigma=0.0, which="LM", tol=1e-12, return_eigenvectors=False)
    assert np.abs(eig[:, None] - lam_ref[None, :]).min(axis=1).max() < 1e-6
    Sg, _, _ = gpu.deflate_get(g)
    S, T = schur.schur_from_eigvecs(lambda q: h @ q, Sg.T)
    assert np.abs(np.tril(S.conj().T @ (h @ S), -1)).max() < 1e-6  # a partial Schur form
    x = synth.gaussian_vectors(12 * v, 2, 55)
    yd = torch.empty((2, 12 * v), dtype=torch.complex128, device=DEV)
    gpu.sign_apply(g, to_dev(x), yd, 80, prec=gpu.F64)
    for r in range(2):
        ref, _ = _schur_ref(h, S, T, x[r], 80)
        assert rel(yd.cpu().numpy()[r], ref) < 1e-11
    g.destroy()


# ------------------------------------- device basis: orthonormality, relation
@pytest.mark.parametrize("prec,otol,rtol", [(0, 1e-12, 1e-12), (1, 1e-5, 1e-5)])
def test_device_basis_orthonormal_and_arnoldi_relation(gpu, prec, otol, rtol):
    """8^4, k = 250, 2 right-hand sides: ||V^H V - I||_max and the Arnoldi
    relation H_w V_k = V_k H_k + h_(k+1,k) v_(k+1) e_k^T (Sec. 4, Eq.
    Arnoldi; Eq. HVAV) for the delayed-reorthogonalisation basis."""
    dims, mu = (8, 8, 8, 8), 0.2
    v = int(np.prod(dims))
    n, k = 12 * v, 250
    links = synth.gauge_links(dims, 3, 0.7)
    h = lattice.hw_operator(links, dims, mu, MW)
    g = gpu.create_gauge_from_links(dims, links, gpu.MIXED)
    gpu.set_mu(g, mu, MW)
    x = synth.gaussian_vectors(n, 2, 81)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    st, info = gpu.sign_apply(g, xd, yd, k, prec=prec)
    for r in range(2):
        V, Hb = gpu.get_krylov(g, r)
        assert V.shape == (k, n) and Hb.shape == (k + 1, k)
        Vk = V.T
        assert np.abs(Vk.conj().T @ Vk - np.eye(k)).max() < otol
        res = h @ Vk - Vk @ Hb[:k, :k]
        hn = np.abs(Hb).max()
        assert np.abs(res[:, : k - 1]).max() < rtol * hn
        # the last column is h_(k+1,k) times a unit vector orthogonal to V_k
        assert abs(np.linalg.norm(res[:, k - 1]) - abs(Hb[k, k - 1])) < rtol * hn
        assert np.abs(Vk.conj().T @ res[:, k - 1]).max() < rtol * hn
    g.destroy()
