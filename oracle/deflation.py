"""LR deflation of critical eigenvalues (Sec. 5.3) and critical eigenpairs.

Right eigenvectors A R_m = R_m Lambda_m (Eq. Rev), left eigenvectors
L_m^H A = Lambda_m L_m^H (Eq. Lev), normalised so that L_m^H R_m = I.
Then x = x_par + x_ominus with x_par = R_m L_m^H x (Eq. xdec), the critical
part is exact, f(A) R_m L_m^H x = R_m f(Lambda_m) L_m^H x (Eq. fARLx), and
the rest goes through Arnoldi on x_ominus (Eq. LRArnoldi):

    f(A) x ~ R_m f(Lambda_m) L_m^H x + beta V_k f(H_k) e_1   (Eq. fAxLRArn)

Reading where the paper allows a choice: the left vectors are
biorthonormalised as L <- L (L^H R)^-H, which makes R L^H the oblique
projector R (L^H R)^-1 L^H also for near-degenerate eigenvalues (the paper
notes that degenerate eigenvalues can be handled by suitable combinations).

Critical eigenvalues: the paper deflates those of smallest magnitude (found
via H_w^2, Sec. 6) as a proxy for smallest |Re lambda|; on the small
lattices the oracle handles it selects smallest |Re lambda| directly from
the full spectrum.
"""

import numpy as np
import scipy.sparse.linalg as spla

from .arnoldi import arnoldi_sign, arnoldi_sign_adaptive
from .signfun import eig_decomposition, sgn_re


def biorthonormalise(r, l):
    """Return L (L^H R)^-H so that the result satisfies L^H R = I."""
    g = l.conj().T @ r
    return l @ np.linalg.inv(g).conj().T


def lr_split(x, r, l_bi):
    """c = L^H x, x_ominus = x - R c (Eq. xdec)."""
    c = l_bi.conj().T @ x
    return c, x - r @ c


def lr_sign_apply(matvec, x, r, l, lam, k, **newton_kw):
    """sgn(A) x by LR deflation + Arnoldi (Eq. fAxLRArn with f = sgn).

    ``r``, ``l``: N x m right/left eigenvector matrices (any normalisation;
    they are biorthonormalised here), ``lam``: the m eigenvalues.
    Returns (y, info); info has k_used, beta, newton_iters, c.
    """
    x = np.asarray(x, dtype=np.complex128)
    m = 0 if r is None else r.shape[1]
    if m == 0:
        y, info = arnoldi_sign(matvec, x, k, **newton_kw)
        info["c"] = np.zeros(0, np.complex128)
        return y, info
    l_bi = biorthonormalise(r, l)
    c, x_om = lr_split(x, r, l_bi)
    y_defl = r @ (sgn_re(lam) * c)
    y_kr, info = arnoldi_sign(matvec, x_om, k, **newton_kw)
    info["c"] = c
    return y_defl + y_kr, info


def lr_sign_apply_adaptive(matvec, x, r, l, lam, k_max, every, tol, skip_ahead=False, **newton_kw):
    """LR deflation (Eq. fAxLRArn) whose Krylov part stops by the convergence
    estimate of ``arnoldi_sign_adaptive`` (the batched form's per-vector stop,
    not in the paper; ``skip_ahead`` selects its skip-ahead check schedule):
    the deflated part is exact, so the estimate is taken
    on the Krylov coefficients of x_ominus. Returns (y, info) as
    ``lr_sign_apply``, with info["k_used"] the step of the stop."""
    x = np.asarray(x, dtype=np.complex128)
    if r is None or r.shape[1] == 0:
        y, info = arnoldi_sign_adaptive(matvec, x, k_max, every, tol, skip_ahead, **newton_kw)
        info["c"] = np.zeros(0, np.complex128)
        return y, info
    l_bi = biorthonormalise(r, l)
    c, x_om = lr_split(x, r, l_bi)
    y_kr, info = arnoldi_sign_adaptive(matvec, x_om, k_max, every, tol, skip_ahead, **newton_kw)
    info["c"] = c
    return r @ (sgn_re(lam) * c) + y_kr, info


def critical_pairs_dense(a, m, decomposition=None):
    """m eigenpairs of smallest |Re lambda| from the full spectrum.

    Returns (lam, R, L) with L^H R = I (L from the rows of U^-1).
    """
    if decomposition is None:
        decomposition = eig_decomposition(a)
    lam, u = decomposition
    order = np.argsort(np.abs(np.real(lam)), kind="stable")[:m]
    uinv = np.linalg.inv(u)
    r = u[:, order]
    l = uinv[order, :].conj().T
    return lam[order], r, l


def critical_pairs_sparse(h_mu, h_minus_mu, m, extra=None, tol=1e-13):
    """Critical pairs of a large sparse H_w(mu) by shift-invert Arnoldi.

    Right vectors: eigenvalues of H_w(mu) nearest 0 (scipy ARPACK, sigma=0);
    left vectors: right eigenvectors of H_w(mu)^H = H_w(-mu) (gamma5-
    hermiticity), whose eigenvalues are the conjugates. m + extra pairs are
    found, the m with smallest |Re lambda| kept, left and right matched by
    eigenvalue, and L biorthonormalised against R.
    """
    if extra is None:
        extra = max(2, m // 2)
    nev = m + extra
    lam_r, vr = spla.eigs(h_mu.tocsc(), k=nev, sigma=0.0, which="LM", tol=tol)
    lam_l, vl = spla.eigs(h_minus_mu.tocsc(), k=nev, sigma=0.0, which="LM", tol=tol)
    order = np.argsort(np.abs(np.real(lam_r)), kind="stable")[:m]
    lam = lam_r[order]
    r = vr[:, order]
    l = np.empty_like(r)
    for i, z in enumerate(lam):
        j = int(np.argmin(np.abs(np.conj(lam_l) - z)))
        l[:, i] = vl[:, j]
    return lam, r, biorthonormalise(r, l)


def sgn_of_eigs(lam):
    """f(lambda_i) = sgn(Re lambda_i) (Sec. 5.3, step ii)."""
    return sgn_re(lam)
