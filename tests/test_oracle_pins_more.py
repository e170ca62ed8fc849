"""Pins of the oracle's critical pairs, Schur deflation with the App. A
Sylvester solver, the harmonic variant and the overlap operator.

Each function is checked against something other than itself: the dense
spectral decomposition, scipy's Sylvester solver, the spectral sign of the
composite Hessenberg matrix, the Petrov-Galerkin definition of harmonic
Ritz values, the Ginsparg-Wilson relation and a dense linear solve. Planted
mistakes (in memory, on the CPU) show that the pins catch the plausible
errors.
"""

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse.linalg

import synth
from oracle import arnoldi, deflation, lattice, overlap, schur, signfun

MW = -1.5


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _problem(dims, seed=1, eps=0.5, mu=0.3):
    u = synth.gauge_links(dims, seed, eps)
    h = lattice.hw_operator(u, dims, mu, MW)
    hm = lattice.hw_operator(u, dims, -mu, MW)
    return h, hm, h.shape[0]


def _mutant(module, old, new):
    import importlib
    import types
    mod = importlib.import_module(f"oracle.{module}")
    src = open(mod.__file__).read()
    assert src.count(old) >= 1, old
    m = types.ModuleType(f"mutant_{module}")
    m.__package__ = "oracle"
    exec(compile(src.replace(old, new, 1), mod.__file__, "exec"), m.__dict__)
    return m


# ------------------------------------------------- critical pairs (Sec. 6)
def _dense_selection(hd, m, extra):
    """The selection rule of critical_pairs_sparse applied to the full
    spectrum: the m + extra eigenvalues of smallest |lambda|, of which the m
    of smallest |Re lambda|, with the spectral projector onto them."""
    lam, u = np.linalg.eig(hd)
    near = np.argsort(np.abs(lam), kind="stable")[: m + extra]
    sel = near[np.argsort(np.abs(lam[near].real), kind="stable")[:m]]
    uinv = np.linalg.inv(u)
    return lam[sel], u[:, sel] @ uinv[sel, :]


@pytest.mark.parametrize("dims,mu", [((2, 4, 4, 4), 0.3), ((2, 2, 4, 4), 0.2)])
def test_critical_pairs_sparse_against_dense(dims, mu):
    """Same eigenvalues (as complex numbers), residuals of Eqs. Rev and Lev,
    L^H R = I and the same spectral projector R L^H as the dense route."""
    h, hm, n = _problem(dims, mu=mu)
    m, extra = 12, 6
    lam, r, l = deflation.critical_pairs_sparse(h, hm, m, extra=extra)
    lam_ref, proj_ref = _dense_selection(h.toarray(), m, extra)
    d = np.abs(lam[:, None] - lam_ref[None, :])
    assert d.min(axis=1).max() < 1e-10 and d.min(axis=0).max() < 1e-10
    hn = np.abs(scipy.sparse.linalg.norm(h, 1))
    assert np.abs(h @ r - r * lam).max() < 1e-10 * hn                       # Eq. Rev
    assert np.abs(l.conj().T @ h - lam[:, None] * l.conj().T).max() < 1e-9 * hn  # Eq. Lev
    assert np.abs(l.conj().T @ r - np.eye(m)).max() < 1e-10
    assert np.abs(r @ l.conj().T - proj_ref).max() < 1e-9


def test_critical_pairs_pin_catches_planted_mismatch():
    """Matching left to right vectors by lambda instead of conj(lambda)."""
    h, hm, n = _problem((2, 4, 4, 4), mu=0.3)
    bad = _mutant("deflation", "np.abs(np.conj(lam_l) - z)", "np.abs(lam_l - z)")
    _, proj_ref = _dense_selection(h.toarray(), 12, 6)
    # mismatched partners either leave L^H R singular (biorthonormalisation
    # fails) or give a wrong spectral projector: both expose the mistake
    try:
        lam, r, l = bad.critical_pairs_sparse(h, hm, 12, extra=6)
    except np.linalg.LinAlgError:
        return
    assert np.abs(r @ l.conj().T - proj_ref).max() > 1e-6


# ---------------------------------------- Sylvester solver (App. A)
def _tri_hess(m, n, seed):
    """T upper triangular with eigenvalues in the left half plane, H the
    Arnoldi Hessenberg matrix of a random matrix with its spectrum around
    2 (disjoint spectra: the Sylvester equation is well posed)."""
    rng = np.random.default_rng(seed)
    t = np.triu(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))) * 0.3
    t[np.diag_indices(m)] = rng.uniform(-3, -1, m) + 0.2j * rng.standard_normal(m)
    a = 2.0 * np.eye(n + 1) + 0.5 * (rng.standard_normal((n + 1, n + 1))
                                     + 1j * rng.standard_normal((n + 1, n + 1))) / np.sqrt(n + 1)
    _, hb, _, ku = arnoldi.arnoldi(lambda q: a @ q, rng.standard_normal(n + 1) + 0j, n)
    assert ku == n
    c = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    return t, hb[:n, :n], c


@pytest.mark.parametrize("m,n", [(1, 1), (5, 7), (12, 40), (30, 3)])
def test_sylvester_against_scipy(m, n):
    """The first column, the only one Eq. formula uses, close to rounding.
    The other columns only for small n: the recurrences of Eq. abij grow
    like a product of |T_ii - H_jj| / |H_(j+1,j)|, so y_ij = a_j y_i1 + b_j
    cancels catastrophically at large j (by n = 40 here the last columns
    are meaningless), while y_i1 stays accurate."""
    t, h, c = _tri_hess(m, n, m * 100 + n)
    y = schur.sylvester_rowwise(t, h, c)
    ref = scipy.linalg.solve_sylvester(t, -h, c)
    assert rel(y[:, 0], ref[:, 0]) < 1e-9
    if n <= 10:
        assert rel(y, ref) < 1e-9


def test_sylvester_pin_catches_planted_mistake():
    t, h, c = _tri_hess(6, 9, 3)
    bad = _mutant("schur", "ct = c[i] - t[i, i + 1:] @ y[i + 1:]", "ct = c[i] + t[i, i + 1:] @ y[i + 1:]")
    ref = scipy.linalg.solve_sylvester(t, -h, c)
    assert rel(bad.sylvester_rowwise(t, h, c)[:, 0], ref[:, 0]) > 1e-3


# ------------------------------------------------ Schur deflation (Sec. 5.2)
def _schur_setup(hd, m, dec=None):
    if dec is None:
        dec = np.linalg.eig(hd)
    lam, u = dec
    order = np.argsort(np.abs(lam.real), kind="stable")[:m]
    s, t = schur.schur_from_eigvecs(lambda q: hd @ q, u[:, order])
    return s, t, lam[order]


def test_schur_basis_is_partial_schur_form():
    """A S = S T (Eq. pSd), S orthonormal, T upper triangular with the
    eigenvalues on its diagonal."""
    h, _, n = _problem((2, 2, 2, 4))
    hd = h.toarray()
    s, t, lam = _schur_setup(hd, 14)
    assert np.abs(s.conj().T @ s - np.eye(14)).max() < 1e-13
    assert np.abs(hd @ s - s @ t).max() < 1e-12
    assert np.allclose(np.tril(t, -1), 0.0)
    assert np.abs(np.diag(t) - lam).max() < 1e-12


def test_modified_arnoldi_composite_relation():
    """Q^H A Q = [[T, X], [0, H_k]] (Eqs. modArnoldi, newH, newHQHQ) with
    Q = (S, V_k) orthonormal."""
    h, _, n = _problem((2, 2, 2, 4))
    hd = h.toarray()
    s, t, _ = _schur_setup(hd, 10)
    x = synth.gaussian_vectors(n, 1, 2)[0]
    xp = x - s @ (s.conj().T @ x)
    k = 40
    v, hh, xx, beta, ku = schur.modified_arnoldi(lambda q: hd @ q, xp, s, k)
    assert ku == k
    q = np.hstack([s, v[:, :k]])
    assert np.abs(q.conj().T @ q - np.eye(10 + k)).max() < 1e-13
    comp = np.block([[t, xx], [np.zeros((k, 10)), hh[:k, :k]]])
    assert np.abs(q.conj().T @ hd @ q - comp).max() < 1e-12
    # A Q = Q H + beta_k v_(k+1) e_(m+k)^T (Eq. modArnoldi)
    resid = hd @ q - q @ comp
    resid[:, -1] -= hh[k, k - 1] * v[:, k]
    assert np.abs(resid).max() < 1e-12


def test_sylvester_block_is_sign_of_composite():
    """The first column of Y equals that of the upper-right block of sgn(H)
    for the composite H (Eq. f_H), sgn taken by the spectral definition
    (Eq. fA)."""
    h, _, n = _problem((2, 2, 2, 4))
    hd = h.toarray()
    s, t, _ = _schur_setup(hd, 8)
    x = synth.gaussian_vectors(n, 1, 3)[0]
    y, info = schur.schur_sign_apply(lambda q: hd @ q, x, s, t, 30)
    k = info["k_used"]
    comp = np.block([[t, info["X"]], [np.zeros((k, 8)), info["H"][:k, :k]]])
    sg = signfun.sgn_matrix(comp)
    assert rel(info["Y"][:, 0], sg[:8, 8]) < 1e-9
    assert rel(info["coeff_v"], info["beta"] * sg[8:, 8]) < 1e-9


def test_schur_full_krylov_is_exact():
    h, _, n = _problem((2, 2, 2, 2))
    hd = h.toarray()
    s, t, _ = _schur_setup(hd, 20)
    x = synth.gaussian_vectors(n, 1, 4)[0]
    y, info = schur.schur_sign_apply(lambda q: hd @ q, x, s, t, n - 20)
    assert rel(y, signfun.sgn_apply_dense(hd, x)) < 1e-10


def test_schur_full_deflation_is_exact():
    h, _, n = _problem((2, 2, 2, 2))
    hd = h.toarray()
    s, t, _ = _schur_setup(hd, n)
    x = synth.gaussian_vectors(n, 1, 5)[0]
    y, info = schur.schur_sign_apply(lambda q: hd @ q, x, s, t, 5)
    assert info["beta"] < 1e-10
    assert rel(y, signfun.sgn_apply_dense(hd, x)) < 1e-10


def test_schur_deflation_improves_and_tracks_lr():
    """Sec. 6: at fixed k the error falls as m grows; Schur and LR deflation
    give errors of the same size (Sec. 5.4; the paper finds LR slightly
    more accurate)."""
    h, hm, n = _problem((2, 2, 2, 4))
    hd = h.toarray()
    dec = np.linalg.eig(hd)
    x = synth.gaussian_vectors(n, 1, 2)[0]
    ref = signfun.sgn_apply_dense(hd, x, dec)
    errs_s, errs_lr = [], []
    for m in (4, 16, 40):
        s, t, _ = _schur_setup(hd, m, dec)
        ys, _ = schur.schur_sign_apply(lambda q: hd @ q, x, s, t, 40)
        lam, r, l = deflation.critical_pairs_dense(hd, m, dec)
        yl, _ = deflation.lr_sign_apply(lambda q: hd @ q, x, r, l, lam, 40)
        errs_s.append(rel(ys, ref))
        errs_lr.append(rel(yl, ref))
    assert errs_s[0] > errs_s[1] > errs_s[2]
    for a, b in zip(errs_s, errs_lr):
        assert 0.1 < a / b < 10.0


def test_schur_pin_catches_planted_mistake():
    h, _, n = _problem((2, 2, 2, 2))
    hd = h.toarray()
    s, t, _ = _schur_setup(hd, 20)
    x = synth.gaussian_vectors(n, 1, 4)[0]
    bad = _mutant("schur", "cc = f_t @ xx - xx @ f_h", "cc = f_t @ xx + xx @ f_h")
    y, _ = bad.schur_sign_apply(lambda q: hd @ q, x, s, t, n - 20)
    assert rel(y, signfun.sgn_apply_dense(hd, x)) > 1e-3


# ------------------------------------------------- harmonic variant (Sec. 4)
@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_harmonic_ritz_values_by_definition(mu):
    """eig(H^_k) are the theta of the Petrov-Galerkin condition
    (A V y - theta V y) orthogonal to A V, solved as a generalised
    eigenproblem on the explicit A V."""
    h, _, n = _problem((2, 2, 2, 4), mu=mu)
    x = synth.gaussian_vectors(n, 1, 2)[0]
    k = 25
    v, hb, beta, ku = arnoldi.arnoldi(lambda q: h @ q, x, k)
    av = h @ v[:, :k]
    theta_ref = scipy.linalg.eigvals(av.conj().T @ av, av.conj().T @ v[:, :k])
    theta = np.linalg.eigvals(arnoldi.harmonic_matrix(hb))
    d = np.abs(theta[:, None] - theta_ref[None, :])
    assert d.min(axis=1).max() < 1e-9 * np.abs(theta_ref).max()
    assert d.min(axis=0).max() < 1e-9 * np.abs(theta_ref).max()


def test_harmonic_removes_see_saw():
    """Sec. 4: with harmonic Ritz values the error no longer alternates
    between odd and even k; plain Arnoldi does."""
    h, _, n = _problem((2, 2, 2, 4))
    x = synth.gaussian_vectors(n, 1, 2)[0]
    ref = signfun.sgn_apply_dense(h.toarray(), x)
    mv = lambda q: h @ q
    plain = [rel(arnoldi.arnoldi_sign(mv, x, k)[0], ref) for k in range(30, 38)]
    harm = [rel(arnoldi.arnoldi_sign(mv, x, k, harmonic=True)[0], ref) for k in range(30, 38)]
    assert min(plain[i + 1] / plain[i] for i in range(0, 7, 2)) > 1.5   # odd k much worse
    assert all(harm[i + 1] <= harm[i] * 1.01 for i in range(7))       # smooth, non-increasing


def test_harmonic_exact_at_full_dimension_and_deflated():
    h, hm, n = _problem((2, 2, 2, 2))
    hd = h.toarray()
    x = synth.gaussian_vectors(n, 1, 9)[0]
    ref = signfun.sgn_apply_dense(hd, x)
    y, _ = arnoldi.arnoldi_sign(lambda q: h @ q, x, n, harmonic=True)
    assert rel(y, ref) < 1e-10
    lam, r, l = deflation.critical_pairs_dense(hd, 20)
    y, _ = deflation.lr_sign_apply(lambda q: h @ q, x, r, l, lam, n - 20, harmonic=True)
    assert rel(y, ref) < 1e-10


def test_harmonic_pin_catches_planted_mistake():
    h, _, n = _problem((2, 2, 2, 4), mu=0.3)
    x = synth.gaussian_vectors(n, 1, 2)[0]
    v, hb, beta, ku = arnoldi.arnoldi(lambda q: h @ q, x, 25)
    av = h @ v[:, :25]
    theta_ref = scipy.linalg.eigvals(av.conj().T @ av, av.conj().T @ v[:, :25])
    bad = _mutant("arnoldi", "f = np.linalg.solve(hk.conj().T, ek)", "f = np.linalg.solve(hk, ek)")
    theta = np.linalg.eigvals(bad.harmonic_matrix(hb))
    d = np.abs(theta[:, None] - theta_ref[None, :])
    assert d.min(axis=1).max() > 1e-6


# ------------------------------------------------- overlap operator (Sec. 2)
@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_ginsparg_wilson_relation(mu):
    """{D_ov, gamma5} = D_ov gamma5 D_ov (Eq. GW:eq) from sgn^2 = 1."""
    h, _, n = _problem((2, 2, 2, 4), mu=mu)
    d = overlap.dov_dense(signfun.sgn_matrix(h.toarray()))
    g5 = np.diag(lattice.gamma5_diag(n // 12)).astype(np.complex128)
    assert np.abs(d @ g5 + g5 @ d - d @ g5 @ d).max() < 1e-11
    # replacing sgn by the polar factor breaks it at mu != 0 (Sec. 2)
    dp = overlap.dov_dense(signfun.polar_factor(h.toarray()))
    gw = np.abs(dp @ g5 + g5 @ dp - dp @ g5 @ dp).max()
    assert (gw < 1e-11) if mu == 0.0 else (gw > 1e-4)


def test_overlap_mu_zero_spectrum_on_circle():
    """At mu = 0, D_ov - 1 = gamma5 sgn(H_w) is unitary: eigenvalues of D_ov
    lie on |z - 1| = 1."""
    h, _, n = _problem((2, 2, 2, 2), mu=0.0)
    d = overlap.dov_dense(signfun.sgn_matrix(h.toarray()))
    z = np.linalg.eigvals(d)
    assert np.abs(np.abs(z - 1.0) - 1.0).max() < 1e-11


def test_dov_apply_matches_dense():
    h, _, n = _problem((2, 2, 2, 4))
    hd = h.toarray()
    sg = signfun.sgn_matrix(hd)
    x = synth.gaussian_vectors(n, 1, 6)[0]
    assert rel(overlap.dov_apply(lambda q: sg @ q, x), overlap.dov_dense(sg) @ x) < 1e-13


@pytest.mark.parametrize("restart", [5, 60])
def test_gmres_against_dense_solve(restart):
    rng = np.random.default_rng(4)
    n = 60
    a = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.2 + 1j * rng.standard_normal((n, n)) * 0.2
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = overlap.gmres(lambda q: a @ q, b, restart, 1e-12, 200)
    assert info["converged"] and info["rel_resid"] <= 1e-12
    assert rel(x, np.linalg.solve(a, b)) < 1e-10
    assert (info["cycles"] > 1) == (restart == 5)


def test_overlap_solve_matches_dense():
    """Nested inversion: GMRES on D_ov x = b with the exact sign equals the
    dense solve."""
    h, _, n = _problem((2, 2, 2, 2), mu=0.3)
    sg = signfun.sgn_matrix(h.toarray())
    b = synth.gaussian_vectors(n, 1, 8)[0]
    x, info = overlap.gmres(lambda q: overlap.dov_apply(lambda z: sg @ z, q), b, 30, 1e-11, 50)
    assert info["converged"]
    assert rel(x, np.linalg.solve(overlap.dov_dense(sg), b)) < 1e-9


def test_gmres_pin_catches_planted_mistake():
    rng = np.random.default_rng(4)
    n = 40
    a = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.2
    b = rng.standard_normal(n) + 0j
    bad = _mutant("overlap", "rhs[0] = beta", "rhs[0] = -beta")
    x, info = bad.gmres(lambda q: a @ q, b, 10, 1e-12, 5)
    assert not info["converged"] or rel(x, np.linalg.solve(a, b)) > 1e-3


# ------------------------------- skip-ahead check schedule (batched form)
def _skip_problem():
    dims = (4, 4, 4, 4)
    u = synth.gauge_links(dims, 3, 0.5)
    h = lattice.hw_operator(u, dims, 0.3, MW)
    return h, synth.gaussian_vectors(h.shape[0], 1, 2)[0]


def _check_schedule(mod, h, x, tol):
    """Invariants of the skip-ahead schedule against checking every interval
    on the same problem (whose convergence slows down, so the extrapolation
    never overshoots): the same stop, fewer sign computations, all on
    multiples of the interval, and the result of the fixed-k method at the
    stop, where the change against the previous check is below tol."""
    mv = lambda q: h @ q
    y, info = mod.arnoldi_sign_adaptive(mv, x, 300, 10, tol, skip_ahead=True)
    _, fixed = arnoldi.arnoldi_sign_adaptive(mv, x, 300, 10, tol)
    ch = info["checks"]
    assert ch[:3] == [10, 20, 30] and all(j % 10 == 0 for j in ch) and ch == sorted(set(ch))
    assert len(ch) < len(fixed["checks"])
    assert info["k_used"] == fixed["k_used"]
    y_fix, at = arnoldi.arnoldi_sign(mv, x, info["k_used"])
    assert np.linalg.norm(y - y_fix) < 1e-13 * np.linalg.norm(y_fix)
    if info["k_used"] < 300:
        _, before = arnoldi.arnoldi_sign(mv, x, ch[-2])
        c = at["coeff"]
        cb = np.zeros_like(c)
        cb[: before["coeff"].shape[0]] = before["coeff"]
        assert np.linalg.norm(c - cb) < tol * np.linalg.norm(c)


@pytest.mark.parametrize("tol", [1e-3, 1e-5, 1e-8])
def test_skip_ahead_schedule(tol):
    h, x = _skip_problem()
    _check_schedule(arnoldi, h, x, tol)


@pytest.mark.parametrize("old,new", [("np.log(e1 / e0)", "np.log(e0 / e1)"),
                                     ("j - j_prev == every", "j - j_prev >= every")])
def test_skip_ahead_pin_catches_planted_mistake(old, new):
    """A flipped rate (no skipping at all) and rates taken from estimates
    over more than one interval (late stops) each break an invariant."""
    h, x = _skip_problem()
    bad = _mutant("arnoldi", old, new)
    with pytest.raises(AssertionError):
        for tol in (1e-3, 1e-5):
            _check_schedule(bad, h, x, tol)
