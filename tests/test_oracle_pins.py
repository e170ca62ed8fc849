"""Pins of the CPU oracle against facts fixed by the paper and mathematics.

Each test checks the oracle against something other than itself: the
free-field closed form (momentum space, FFT), gauge covariance, gamma5-
hermiticity, the Hermitian mu = 0 case, sgn^2 = I, exactness of Arnoldi at
the grade of x, Newton against scipy.linalg.signm and against matrices with
a known eigen-decomposition, and LR deflation on exact eigenvectors.
"""

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import arnoldi, deflation, freefield, lattice, newton, signfun

MU, MW = 0.3, -1.5


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ---------------------------------------------------------------- gamma basis
def test_gamma_clifford_and_gamma5():
    g = lattice.gamma_matrices()
    for i in range(4):
        assert np.allclose(g[i], g[i].conj().T)
        for j in range(4):
            ac = g[i] @ g[j] + g[j] @ g[i]
            assert np.allclose(ac, 2.0 * (i == j) * np.eye(4))
    assert np.allclose(lattice.gamma5(), np.diag([1, 1, -1, -1]))


def test_kappa():
    assert lattice.kappa_of(-1.5) == pytest.approx(0.2)
    assert lattice.kappa_of(-2.0) == pytest.approx(0.25)


# ------------------------------------------------------- operator: closed form
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 3, 2, 4), (4, 2, 3, 2)])
@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_free_field_operator(dims, mu):
    """Sparse H_w with unit links equals gamma5 D(p) in momentum space."""
    v = int(np.prod(dims))
    h = lattice.hw_operator(synth.unit_links(dims), dims, mu, MW)
    x = synth.gaussian_vectors(12 * v, 1, 11)[0]
    ref = freefield.apply_free(x, dims, mu, MW, "H")
    assert np.abs(h @ x - ref).max() < 1e-13


@pytest.mark.parametrize("mu", [0.0, 0.2])
def test_sampled_sites_pure_gauge_closed_form(mu):
    """H_w x summed at single sites equals Omega H[1] Omega^+ x from the FFT
    closed form: pins the per-site hops, link daggers and the antiperiodic
    wrap (the sampled sites include every face of the lattice)."""
    dims = (4, 6, 2, 8)
    v = int(np.prod(dims))
    u, om = synth.pure_gauge_links(dims, 23)
    x = synth.gaussian_vectors(12 * v, 1, 13)[0]
    ref = freefield.apply_free(x, dims, mu, MW, "H", omega=om).reshape(v, 12)
    rng = np.random.default_rng(3)
    sites = np.unique(np.concatenate([[0, v - 1, 3, 4 * 6 * 2 * 7, 5], rng.integers(0, v, 40)]))
    got = lattice.hw_sites(u, dims, mu, MW, x, sites)
    assert np.abs(got - ref[sites]).max() < 1e-13


def test_sampled_sites_match_sparse_operator():
    """On a random field every site of the per-site sum equals the row of the
    sparse operator, in both hop conventions."""
    dims = (4, 4, 2, 4)
    v = int(np.prod(dims))
    u = synth.gauge_links(dims, 7, 0.6)
    x = synth.gaussian_vectors(12 * v, 1, 14)[0]
    for conv in ("minus_forward", "paper"):
        h = lattice.hw_operator(u, dims, MU, MW, conv)
        got = lattice.hw_sites(u, dims, MU, MW, x, np.arange(v), conv)
        assert np.abs(got.ravel() - h @ x).max() < 1e-13


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
def test_pure_gauge_covariance(dims):
    """H[Omega Omega^+] = Omega H[1] Omega^+ pins link placement and daggers."""
    v = int(np.prod(dims))
    u, om = synth.pure_gauge_links(dims, 21)
    h = lattice.hw_operator(u, dims, MU, MW)
    x = synth.gaussian_vectors(12 * v, 1, 12)[0]
    ref = freefield.apply_free(x, dims, MU, MW, "H", omega=om)
    assert np.abs(h @ x - ref).max() < 1e-13


def test_gauge_covariance_random_field():
    """D[U^Omega] Omega x = Omega D[U] x for a non-trivial field."""
    dims = (2, 2, 2, 4)
    v = 32
    u = synth.gauge_links(dims, 3, 0.7)
    om = synth.random_su3(np.arange(v) + 10_000, 5, 3.0)
    ut = np.empty_like(u)
    for nu in range(4):
        fwd, _ = lattice.neighbour(dims, nu, +1)
        ut[:, nu] = om @ u[:, nu] @ np.conj(np.swapaxes(om[fwd], -1, -2))
    x = synth.gaussian_vectors(12 * v, 1, 4)[0].reshape(v, 4, 3)
    ox = np.einsum("sab,sib->sia", om, x).ravel()
    lhs = lattice.wilson_dirac(ut, dims, MU, MW) @ ox
    dx = (lattice.wilson_dirac(u, dims, MU, MW) @ x.ravel()).reshape(v, 4, 3)
    rhs = np.einsum("sab,sib->sia", om, dx).ravel()
    assert np.abs(lhs - rhs).max() < 1e-13


def test_gamma5_hermiticity():
    """H_w(mu)^dagger = H_w(-mu), i.e. D(mu)^+ = gamma5 D(-mu) gamma5."""
    dims = (2, 2, 2, 4)
    u = synth.gauge_links(dims, 1, 0.5)
    hp = lattice.hw_operator(u, dims, MU, MW).toarray()
    hm = lattice.hw_operator(u, dims, -MU, MW).toarray()
    assert np.abs(hp.conj().T - hm).max() < 1e-15
    assert np.abs(hp - hp.conj().T).max() > 0.1  # non-Hermitian for mu != 0


def test_mu_zero_hermitian():
    dims = (2, 2, 2, 2)
    u = synth.gauge_links(dims, 1, 0.5)
    h0 = lattice.hw_operator(u, dims, 0.0, MW).toarray()
    assert np.abs(h0 - h0.conj().T).max() < 1e-15


def test_hop_conventions_related_by_gamma5():
    """Eq. Dw as printed vs the adopted convention: D_p = g5 D_b g5."""
    dims = (2, 2, 2, 4)
    u = synth.gauge_links(dims, 2, 0.6)
    db = lattice.wilson_dirac(u, dims, MU, MW, "minus_forward").toarray()
    dp = lattice.wilson_dirac(u, dims, MU, MW, "paper").toarray()
    g5 = np.diag(lattice.gamma5_diag(32))
    assert np.abs(dp - g5 @ db @ g5).max() < 1e-15
    hb = g5 @ db
    hp = g5 @ dp
    sb = signfun.sgn_matrix(hb)
    sp_ = signfun.sgn_matrix(hp)
    assert np.abs(sp_ - g5 @ sb @ g5).max() < 1e-11


def test_extent_two_hops_add():
    """On an extent-2 axis the forward and backward neighbours coincide; both
    hops must still be present (checked against the closed form)."""
    dims = (2, 2, 2, 2)
    d = lattice.wilson_dirac(synth.unit_links(dims), dims, 0.0, MW)
    x = np.ones(12 * 16, dtype=np.complex128)
    y = d @ x
    ref = freefield.apply_free(x, dims, 0.0, MW, "D")
    assert np.abs(y - ref).max() < 1e-13


# ----------------------------------------------------------- spectral sign
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
def test_sign_free_field_closed_form(dims):
    v = int(np.prod(dims))
    h = lattice.hw_operator(synth.unit_links(dims), dims, MU, MW).toarray()
    x = synth.gaussian_vectors(12 * v, 1, 5)[0]
    ref = freefield.apply_free(x, dims, MU, MW, "sgnH")
    assert np.abs(signfun.sgn_apply_dense(h, x) - ref).max() < 1e-12


def test_sign_pure_gauge_closed_form():
    dims = (2, 2, 2, 4)
    u, om = synth.pure_gauge_links(dims, 8)
    h = lattice.hw_operator(u, dims, MU, MW).toarray()
    x = synth.gaussian_vectors(384, 1, 6)[0]
    ref = freefield.apply_free(x, dims, MU, MW, "sgnH", omega=om)
    assert np.abs(signfun.sgn_apply_dense(h, x) - ref).max() < 1e-12


def test_sign_invariants_random_field():
    dims = (2, 2, 2, 4)
    u = synth.gauge_links(dims, 1, 0.5)
    h = lattice.hw_operator(u, dims, MU, MW).toarray()
    s = signfun.sgn_matrix(h)
    assert np.abs(s @ s - np.eye(384)).max() < 1e-11  # Sec. 2: sgn(A)^2 = I
    assert np.abs(s @ h - h @ s).max() < 1e-11  # f(H) H = H f(H)
    # sgn(H(mu))^dagger = sgn(H(-mu)) from gamma5-hermiticity
    hm = lattice.hw_operator(u, dims, -MU, MW).toarray()
    assert np.abs(s.conj().T - signfun.sgn_matrix(hm)).max() < 1e-11
    # Ginsparg-Wilson relation of D_ov = 1 + gamma5 sgn(H) (Eq. GW)
    g5 = np.diag(lattice.gamma5_diag(32))
    dov = np.eye(384) + g5 @ s
    assert np.abs(dov @ g5 + g5 @ dov - dov @ g5 @ dov).max() < 1e-11


def test_sign_equals_polar_only_for_hermitian():
    """Sec. 2: pol(A) = sgn(A) iff A Hermitian (here: mu = 0 vs mu != 0)."""
    dims = (2, 2, 2, 2)
    u = synth.gauge_links(dims, 1, 0.5)
    h0 = lattice.hw_operator(u, dims, 0.0, MW).toarray()
    lam, q = np.linalg.eigh(h0)
    s_eigh = q @ np.diag(np.sign(lam)) @ q.conj().T
    assert np.abs(signfun.sgn_matrix(h0) - s_eigh).max() < 1e-11
    assert np.abs(signfun.polar_factor(h0) - s_eigh).max() < 1e-11
    h = lattice.hw_operator(u, dims, 0.5, MW).toarray()
    pol = signfun.polar_factor(h)
    assert np.abs(signfun.sgn_matrix(h) - pol).max() > 1e-3
    assert np.abs(pol @ pol - np.eye(192)).max() > 1e-3


def test_sgn_scalar():
    z = np.array([1 + 2j, -0.1 + 5j, -3 - 1j, 0.2 - 9j])
    assert np.allclose(signfun.sgn_scalar(z), [1, -1, -1, 1])
    with pytest.raises(ValueError):
        signfun.sgn_re(np.array([1j]))


# ------------------------------------------------------------------- Newton
def _known_matrix(n, seed, gap=0.2):
    rng = np.random.default_rng(seed)
    re = rng.uniform(gap, 3.0, n) * np.where(rng.random(n) < 0.5, -1, 1)
    lam = re + 1j * rng.uniform(-1, 1, n)
    u = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return u @ np.diag(lam) @ np.linalg.inv(u), u @ np.diag(np.sign(re)) @ np.linalg.inv(u)


@pytest.mark.parametrize("n", [1, 5, 40])
def test_newton_known_decomposition(n):
    a, s_ref = _known_matrix(n, n)
    s, it = newton.roberts_sign(a)
    assert rel(s, s_ref) < 1e-10
    assert it < 50


def test_newton_vs_signm_hessenberg():
    a, _ = _known_matrix(30, 7)
    h = scipy.linalg.hessenberg(a)
    s, _ = newton.roberts_sign(h)
    assert rel(s, scipy.linalg.signm(h)) < 1e-9
    assert np.abs(s @ s - np.eye(30)).max() < 1e-10


def test_newton_fails_on_imaginary_axis():
    a = np.diag([1.0, 1j])
    with pytest.raises((newton.NewtonNotConverged, np.linalg.LinAlgError)):
        newton.roberts_sign(a, max_iter=30)


# ------------------------------------------------------------------ Arnoldi
def _small_problem(dims=(2, 2, 2, 4), seed=1, eps=0.5, mu=MU):
    v = int(np.prod(dims))
    u = synth.gauge_links(dims, seed, eps)
    h = lattice.hw_operator(u, dims, mu, MW)
    return h, 12 * v


def test_arnoldi_orthonormal_and_relation():
    h, n = _small_problem()
    x = synth.gaussian_vectors(n, 1, 2)[0]
    k = 60
    v, hh, beta, ku = arnoldi.arnoldi(lambda q: h @ q, x, k)
    assert ku == k
    assert np.abs(v.conj().T @ v - np.eye(k + 1)).max() < 1e-13
    resid = h @ v[:, :k] - v @ hh
    assert np.abs(resid).max() < 1e-13
    assert np.allclose(np.tril(hh, -2), 0)
    assert beta == pytest.approx(1.0)


def test_arnoldi_exact_at_full_dimension():
    h, n = _small_problem()
    x = synth.gaussian_vectors(n, 1, 9)[0]
    y, info = arnoldi.arnoldi_sign(lambda q: h @ q, x, n)
    ref = signfun.sgn_apply_dense(h.toarray(), x)
    assert rel(y, ref) < 1e-11


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (8, 8, 8, 16)])
def test_arnoldi_breakdown_at_grade_free_field(dims):
    """Two plane waves: grade <= 4, Arnoldi stops early and is exact."""
    h = lattice.hw_operator(synth.unit_links(dims), dims, MU, MW)
    x = synth.plane_wave_vectors(dims, [(1, 0, 0, 0), (0, 2, 1, 3)], 7)[0]
    y, info = arnoldi.arnoldi_sign(lambda q: h @ q, x, 30)
    assert info["k_used"] <= 4
    ref = freefield.apply_free(x, dims, MU, MW, "sgnH")
    assert rel(y, ref) < 1e-12


def test_arnoldi_zero_vector():
    h, n = _small_problem()
    y, info = arnoldi.arnoldi_sign(lambda q: h @ q, np.zeros(n, np.complex128), 10)
    assert info["k_used"] == 0 and np.all(y == 0)


def test_even_odd_see_saw_converges():
    """Sec. 4: the error oscillates between odd and even k but falls."""
    h, n = _small_problem()
    x = synth.gaussian_vectors(n, 1, 2)[0]
    ref = signfun.sgn_apply_dense(h.toarray(), x)
    errs = [rel(arnoldi.arnoldi_sign(lambda q: h @ q, x, k)[0], ref) for k in (40, 80, 160, 240)]
    assert errs[-1] < errs[0]


# ---------------------------------------------------------------- deflation
def test_lr_deflation_exact_eigvec():
    """x = r_i: x_ominus = 0, y = sgn(lambda_i) r_i exactly (Eq. fARLx)."""
    h, n = _small_problem()
    hd = h.toarray()
    lam, r, l = deflation.critical_pairs_dense(hd, 10)
    for i in (0, 3, 9):
        y, info = deflation.lr_sign_apply(lambda q: h @ q, r[:, i], r, l, lam, 20)
        assert info["beta"] < 1e-12
        assert rel(y, np.sign(lam[i].real) * r[:, i]) < 1e-12


def test_lr_biorthonormal_and_projector():
    h, n = _small_problem()
    lam, r, l = deflation.critical_pairs_dense(h.toarray(), 12)
    hd = h.toarray()
    assert np.abs(hd @ r - r * lam).max() < 1e-12  # Eq. Rev
    assert np.abs(l.conj().T @ hd - lam[:, None] * l.conj().T).max() < 1e-12  # Eq. Lev
    # rescaled, non-biorthonormal left vectors are fixed by biorthonormalise
    lb = deflation.biorthonormalise(r, l * (0.3 + 2j))
    assert np.abs(lb.conj().T @ r - np.eye(12)).max() < 1e-12


def test_lr_full_deflation_is_exact():
    h, n = _small_problem((2, 2, 2, 2))
    hd = h.toarray()
    lam, r, l = deflation.critical_pairs_dense(hd, n)
    x = synth.gaussian_vectors(n, 1, 3)[0]
    y, info = deflation.lr_sign_apply(lambda q: h @ q, x, r, l, lam, 5)
    assert info["beta"] < 1e-10
    assert rel(y, signfun.sgn_apply_dense(hd, x)) < 1e-10


def test_lr_deflation_improves_convergence():
    """Sec. 6: at fixed k the error falls as m grows."""
    h, n = _small_problem()
    hd = h.toarray()
    dec = signfun.eig_decomposition(hd)
    x = synth.gaussian_vectors(n, 1, 2)[0]
    ref = signfun.sgn_apply_dense(hd, x, dec)
    errs = []
    for m in (0, 10, 40):
        lam, r, l = deflation.critical_pairs_dense(hd, m, dec)
        y, _ = deflation.lr_sign_apply(lambda q: h @ q, x, r if m else None, l, lam, 40)
        errs.append(rel(y, ref))
    assert errs[0] > errs[1] > errs[2]


def test_hermitian_deflation_special_case():
    """mu = 0: left = right eigenvectors, Eq. fAxdefl with orthonormal u_i."""
    h, n = _small_problem(mu=0.0)
    hd = h.toarray()
    lam, q = np.linalg.eigh(hd)
    order = np.argsort(np.abs(lam))[:16]
    u = q[:, order]
    x = synth.gaussian_vectors(n, 1, 5)[0]
    y1, _ = deflation.lr_sign_apply(lambda z: h @ z, x, u, u, lam[order].astype(complex), 60)
    x_perp = x - u @ (u.conj().T @ x)
    y_k, _ = arnoldi.arnoldi_sign(lambda z: h @ z, x_perp, 60)
    y2 = u @ (np.sign(lam[order]) * (u.conj().T @ x)) + y_k
    assert rel(y1, y2) < 1e-12


def test_adaptive_stops_and_matches_fixed_k():
    """The convergence-stopped Arnoldi returns the fixed-k result at its k."""
    h, n = _small_problem()
    x = synth.gaussian_vectors(n, 1, 2)[0]
    y, info = arnoldi.arnoldi_sign_adaptive(lambda q: h @ q, x, 300, 10, 1e-4)
    assert info["k_used"] % 10 == 0 and info["k_used"] < 300 and info["est"] < 1e-4
    y_fix, _ = arnoldi.arnoldi_sign(lambda q: h @ q, x, info["k_used"])
    assert rel(y, y_fix) < 1e-13
    # the estimate tracks the true change: the error vs the dense sign is small
    ref = signfun.sgn_apply_dense(h.toarray(), x)
    assert rel(y, ref) < 1e-2


def test_lr_adaptive_stop_matches_fixed_k_and_exact():
    """The deflated adaptive form equals the fixed-k form at the step where it
    stops, stops earlier than the undeflated adaptive form, and its result
    is within a small multiple of the stopping tolerance of the dense sgn."""
    h, n = _small_problem()
    hd = h.toarray()
    dec = signfun.eig_decomposition(hd)
    x = synth.gaussian_vectors(n, 1, 5)[0]
    ref = signfun.sgn_apply_dense(hd, x, dec)
    lam, r, l = deflation.critical_pairs_dense(hd, 20, dec)
    mv = lambda q: h @ q
    y, info = deflation.lr_sign_apply_adaptive(mv, x, r, l, lam, 300, 10, 1e-8)
    assert info["k_used"] % 10 == 0 and info["est"] < 1e-8
    y_fixed, _ = deflation.lr_sign_apply(mv, x, r, l, lam, info["k_used"])
    assert rel(y, y_fixed) < 1e-13
    _, info0 = deflation.lr_sign_apply_adaptive(mv, x, None, None, None, 300, 10, 1e-8)
    assert info["k_used"] < info0["k_used"]
    assert rel(y, ref) < 1e-6



# ------------------------------------------------ planted mistakes are caught
def _mutant(module, old, new):
    """The module's source with one plausible mistake planted (in memory)."""
    import importlib
    import types
    mod = importlib.import_module(f"oracle.{module}")
    src = open(mod.__file__).read()
    assert src.count(old) >= 1, old
    m = types.ModuleType(f"mutant_{module}")
    m.__package__ = "oracle"
    exec(compile(src.replace(old, new, 1), mod.__file__, "exec"), m.__dict__)
    return m


@pytest.mark.parametrize("old,new", [
    ("u = np.conj(np.swapaxes(links[nb, nu], -1, -2))", "u = links[nb, nu]"),          # missing dagger
    ("bc = np.where(wrapped & (nu == 3), -1.0, 1.0)\n            if step",
     "bc = np.where(wrapped & (nu == 3), 1.0, 1.0)\n            if step"),           # periodic in time
    ("w = 1.0 / tfac", "w = tfac"),                                                  # e^{+mu} backward
    ("proj = one - sign_fwd * gam[nu]\n                u = np.conj",
     "proj = one + sign_fwd * gam[nu]\n                u = np.conj"),               # projector sign
])
def test_stencil_pin_catches_planted_mistakes(old, new):
    dims = (4, 6, 2, 8)
    v = int(np.prod(dims))
    u, om = synth.pure_gauge_links(dims, 23)
    x = synth.gaussian_vectors(12 * v, 1, 13)[0]
    ref = freefield.apply_free(x, dims, 0.2, MW, "H", omega=om).reshape(v, 12)
    bad = _mutant("lattice", old, new).hw_sites(u, dims, 0.2, MW, x, np.arange(v))
    assert np.abs(bad - ref).max() > 1e-6


def test_newton_pin_catches_planted_mistake():
    a = np.diag([2.0, -0.5, 1.5, -3.0]).astype(np.complex128) + 0.1 * np.triu(np.ones((4, 4)), 1)
    bad = _mutant("newton", "s_new = 0.5 * (s + np.linalg.inv(s))", "s_new = 0.5 * (s + np.linalg.inv(s).T)")
    try:
        s, _ = bad.roberts_sign(a)
    except Exception:  # a wrong iteration may not converge at all
        return
    assert np.abs(s - scipy.linalg.signm(a)).max() > 1e-6


def test_deflation_pin_catches_planted_mistake():
    h, n = _small_problem()
    hd = h.toarray()
    dec = signfun.eig_decomposition(hd)
    lam, r, l = deflation.critical_pairs_dense(hd, n, dec)
    x = synth.gaussian_vectors(n, 1, 4)[0]
    ref = signfun.sgn_apply_dense(hd, x, dec)
    bad = _mutant("deflation", "y_defl = r @ (sgn_re(lam) * c)", "y_defl = r @ (np.abs(sgn_re(lam)) * c)")
    y, _ = bad.lr_sign_apply(lambda q: h @ q, x, r, l, lam, 2)
    assert rel(y, ref) > 1e-3
