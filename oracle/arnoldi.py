"""Arnoldi function approximation f(A)x ~ beta V_k f(H_k) e_1.

Arnoldi recurrence A V_k = V_k H_k + beta_k v_(k+1) e_k^T with v_1 = x/beta,
beta = |x| (Sec. 4, Eq. Arnoldi); H_k = V_k^dagger A V_k (Eq. HVAV); the
approximation beta V_k f(H_k) e_1 (Eq. yproj3). With f = sgn, f(H_k) comes
from Roberts' iteration (Sec. 5.2, Eq. Roberts).

Readings where the paper is silent:

* orthogonalisation: classical Gram-Schmidt applied twice (CGS2) per step:
  h1 = V^H w, w -= V h1, h2 = V^H w, w -= V h2, column = h1 + h2;
* breakdown: if H_(j+1,j) <= 1e-12 ||H_(1:j+1,1:j)||_F the Krylov space is
  invariant, the recurrence stops and k_used = j (the result is then exact);
* harmonic variant (the see-saw-free form the paper cites in Sec. 4, from
  harmonic Ritz values): f(H_k) is replaced by f(H^_k) with
  H^_k = H_k + |h_(k+1,k)|^2 H_k^-H e_k e_k^T, whose eigenvalues are the
  harmonic Ritz values of A on K_k (the theta with A V y - theta V y
  orthogonal to A K_k);
* stopping by convergence (batched form; the paper fixes k instead): every
  `every` (even) steps form c_j = beta sgn(H_j) e_1 and stop at the first j
  with ||c_j - c_(j-every)|| / ||c_j|| < tol (c padded with zeros); as V is
  orthonormal this is the relative change of beta V_j sgn(H_j) e_1;
* skip-ahead check schedule (optional; fewer sign computations while the
  estimate is far from tol): the checks fall on multiples of `every`, the
  last one allowed for extrapolation at J = every floor((k_max - 1)/every).
  A check whose previous check lies exactly `every` steps back gives a
  one-interval estimate. After two such estimates e0 (at j0) and e1 (at j1)
  with e1 < e0, the estimate is extrapolated geometrically: it reaches tol
  after n = log(tol/e1) / (log(e1/e0)/(j1 - j0)) more steps, and the checks
  are skipped up to P = every floor((j1 + n)/every) - every (at most
  J - every). The check at P stores c_P (its estimate spans more than one
  interval; it still stops the iteration if below tol) and the check at
  P + every, the last multiple of `every` before the extrapolated stop,
  gives the next one-interval estimate. On a geometric convergence this
  stops at the same j as checking every `every` steps; a convergence that
  speeds up can stop later. Every stop still needs an estimate below tol.
"""

import numpy as np

from .newton import roberts_sign

BREAKDOWN_TOL = 1e-12


def arnoldi(matvec, x, k):
    """Run k Arnoldi steps on x.

    Returns (V, H, beta, k_used): V is N x (k_used+1) (the last column is
    v_(k_used+1), zero after a breakdown), H is (k_used+1) x k_used.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[0]
    beta = np.linalg.norm(x)
    v = np.zeros((n, k + 1), dtype=np.complex128)
    h = np.zeros((k + 1, k), dtype=np.complex128)
    if beta == 0.0 or k == 0:
        return v[:, :1], h[:1, :0], beta, 0
    v[:, 0] = x / beta
    for j in range(k):
        w = matvec(v[:, j])
        basis = v[:, : j + 1]
        h1 = basis.conj().T @ w
        w = w - basis @ h1
        h2 = basis.conj().T @ w
        w = w - basis @ h2
        h[: j + 1, j] = h1 + h2
        hn = np.linalg.norm(w)
        h[j + 1, j] = hn
        if hn <= BREAKDOWN_TOL * np.linalg.norm(h[: j + 2, : j + 1]):
            h[j + 1, j] = 0.0
            return v[:, : j + 2] * np.r_[np.ones(j + 1), 0.0], h[: j + 2, : j + 1], beta, j + 1
        v[:, j + 1] = w / hn
    return v, h, beta, k


def harmonic_matrix(h):
    """H^_k = H_k + |h_(k+1,k)|^2 H_k^-H e_k e_k^T from Hbar_k ((k+1) x k).

    The Petrov-Galerkin condition (A V_k - theta V_k) y orthogonal to A V_k
    with A V_k = V_(k+1) Hbar_k reads Hbar_k^H Hbar_k y = theta H_k^H y, and
    Hbar_k^H Hbar_k = H_k^H H_k + |h_(k+1,k)|^2 e_k e_k^T.
    """
    k = h.shape[1]
    hk = np.array(h[:k, :k], dtype=np.complex128)
    sub = h[k, k - 1] if h.shape[0] > k else 0.0
    if sub == 0.0:
        return hk
    ek = np.zeros(k, dtype=np.complex128)
    ek[-1] = 1.0
    f = np.linalg.solve(hk.conj().T, ek)
    hk[:, -1] += abs(sub) ** 2 * f
    return hk


def arnoldi_sign(matvec, x, k, harmonic=False, **newton_kw):
    """beta V_k sgn(H_k) e_1 (Eq. yproj3 with f = sgn); with ``harmonic``,
    beta V_k sgn(H^_k) e_1 (the harmonic variant above).

    Returns (y, info) with info = dict(k_used, beta, newton_iters, coeff).
    """
    v, h, beta, k_used = arnoldi(matvec, x, k)
    if k_used == 0:
        return np.zeros_like(np.asarray(x, dtype=np.complex128)), dict(
            k_used=0, beta=beta, newton_iters=0, coeff=np.zeros(0, np.complex128))
    hk = harmonic_matrix(h[: k_used + 1, :k_used]) if harmonic else h[:k_used, :k_used]
    s, it = roberts_sign(hk, **newton_kw)
    coeff = beta * s[:, 0]
    y = v[:, :k_used] @ coeff
    return y, dict(k_used=k_used, beta=beta, newton_iters=it, coeff=coeff, H=h)


def arnoldi_sign_adaptive(matvec, x, k_max, every, tol, skip_ahead=False, **newton_kw):
    """Eq. yproj3 with k chosen by the convergence estimate above (with
    ``skip_ahead``, on the skip-ahead schedule).

    Returns (y, info) with info = dict(k_used, est, beta, coeff, checks), where
    checks lists the j at which sgn(H_j) was formed.
    """
    v, h, beta, k_run = arnoldi(matvec, x, k_max)
    cap = every * ((k_max - 1) // every)
    c_prev = np.zeros(0, dtype=np.complex128)
    j_prev = 0
    est = 0.0
    hist = []  # (j, one-interval estimate)
    checks = []
    j = every
    while j <= k_run:
        s, _ = roberts_sign(h[:j, :j], **newton_kw)
        checks.append(j)
        c = beta * s[:, 0]
        prev = np.zeros(j, dtype=np.complex128)
        prev[: c_prev.shape[0]] = c_prev
        est = np.linalg.norm(c - prev) / np.linalg.norm(c)
        if est < tol:
            return v[:, :j] @ c, dict(k_used=j, est=est, beta=beta, coeff=c, checks=checks)
        nxt = j + every
        if skip_ahead and j_prev > 0 and j - j_prev == every:
            hist.append((j, est))
            if len(hist) >= 2 and hist[-1][1] < hist[-2][1]:
                (j0, e0), (j1, e1) = hist[-2], hist[-1]
                n = np.log(tol / e1) / (np.log(e1 / e0) / (j1 - j0))
                t = j1 + n
                p = cap - every if t >= cap else every * int(np.floor(t / every)) - every
                nxt = max(nxt, p)
        c_prev, j_prev = c, j
        j = nxt
    y, info = arnoldi_sign(matvec, x, k_run, **newton_kw)
    info["est"] = est
    info["checks"] = checks
    return y, info
