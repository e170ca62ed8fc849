"""Overlap Dirac operator at chemical potential and its nested inversion.

D_ov(mu) = 1 + gamma5 sgn(H_w(mu)), H_w(mu) = gamma5 D_w(mu) (Sec. 2,
Eq. Dov). Because sgn(A)^2 = 1 for any A, D_ov satisfies the Ginsparg-
Wilson relation {D_ov, gamma5} = D_ov gamma5 D_ov (Sec. 2, Eq. GW:eq).

The paper names the inversion of D_ov by an iterative method whose every
iteration applies sgn(H_w) to a vector, reusing the deflation set-up, as
the use of its method (Secs. 6, 7), and leaves the outer method open.
Reading adopted here: restarted GMRES (the operator is not Hermitian at
mu != 0), zero initial guess, classical Gram-Schmidt applied twice for the
outer basis, the small least-squares problem min ||beta e_1 - Hbar y||
solved by a library routine, a stop inside a cycle once the least-squares
residual is below tol ||b||, and the true residual b - D_ov x recomputed at
the end of every cycle.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""

import numpy as np

from .lattice import gamma5_diag


def dov_apply(sign_apply, x):
    """D_ov x = x + gamma5 sgn(H_w) x (Eq. Dov); ``sign_apply(x)`` returns
    sgn(H_w) x for one vector."""
    x = np.asarray(x, dtype=np.complex128)
    return x + gamma5_diag(x.shape[0] // 12) * sign_apply(x)


def dov_dense(sgn_h):
    """Dense D_ov = 1 + gamma5 sgn(H_w) from the dense sign matrix."""
    n = sgn_h.shape[0]
    g5 = gamma5_diag(n // 12)
    return np.eye(n, dtype=np.complex128) + g5[:, None] * sgn_h


def gmres(apply, b, restart, tol, max_cycles):
    """Restarted GMRES for A x = b with x_0 = 0 (the reading above).

    Returns (x, info) with info = dict(iters (total A applications inside
    cycles), cycles, rel_resid (true, ||b - A x|| / ||b||), converged).
    """
    b = np.asarray(b, dtype=np.complex128)
    n = b.shape[0]
    bnorm = np.linalg.norm(b)
    x = np.zeros(n, dtype=np.complex128)
    if bnorm == 0.0:
        return x, dict(iters=0, cycles=0, rel_resid=0.0, converged=True)
    r = b.copy()
    iters = 0
    rel = 1.0
    for cyc in range(1, max_cycles + 1):
        beta = np.linalg.norm(r)
        w = np.zeros((n, restart + 1), dtype=np.complex128)
        hb = np.zeros((restart + 1, restart), dtype=np.complex128)
        w[:, 0] = r / beta
        y = np.zeros(0, dtype=np.complex128)
        for j in range(restart):
            z = apply(w[:, j])
            iters += 1
            basis = w[:, : j + 1]
            h1 = basis.conj().T @ z
            z = z - basis @ h1
            h2 = basis.conj().T @ z
            z = z - basis @ h2
            hb[: j + 1, j] = h1 + h2
            hn = np.linalg.norm(z)
            hb[j + 1, j] = hn
            rhs = np.zeros(j + 2, dtype=np.complex128)
            rhs[0] = beta
            y = np.linalg.lstsq(hb[: j + 2, : j + 1], rhs, rcond=None)[0]
            ls = np.linalg.norm(rhs - hb[: j + 2, : j + 1] @ y)
            if ls <= tol * bnorm or hn == 0.0:
                break
            w[:, j + 1] = z / hn
        x = x + w[:, : y.shape[0]] @ y
        r = b - apply(x)
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            return x, dict(iters=iters, cycles=cyc, rel_resid=rel, converged=True)
    return x, dict(iters=iters, cycles=max_cycles, rel_resid=rel, converged=False)
