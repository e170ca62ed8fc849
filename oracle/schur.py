"""Schur deflation of critical eigenvalues (Sec. 5.2) and the Sylvester
solver of App. A.

Set-up (Sec. 5.2 steps i-ii): from m right eigenvectors R of A, an
orthonormal basis S_m of their span with A S_m = S_m T_m and T_m upper
triangular (Eq. pSd); T_m = S_m^H A S_m, and f(T_m) by Roberts' iteration.

Application (Sec. 5.2 steps iii-vi):

* x_perp = (1 - S_m S_m^H) x, beta = |x_perp|, v_1 = x_perp / beta;
* modified Arnoldi: every new vector A v_j is orthogonalised against the
  Schur vectors and the previous Arnoldi vectors (Eq. modArnoldi), which
  yields H_k (upper Hessenberg) and X = S_m^H A V_k;
* composite H = [[T_m, X], [0, H_k]] = Q^H A Q with Q = (S_m, V_k)
  (Eqs. newH, newHQHQ), and f(H) = [[f(T_m), Y], [0, f(H_k)]] (Eq. f_H),
  Y solving T_m Y - Y H_k = f(T_m) X - X f(H_k) (Eq. SylvEq);
* f(A) x ~ S_m f(T_m) S_m^H x + (S_m, V_k) (Y; f(H_k)) V_k^H x with
  V_k^H x = beta e_1 (Eq. formula).

Readings where the paper leaves a choice:

* orthogonalisation: classical Gram-Schmidt applied twice against the
  composite basis (S_m, V_j), as in the oracle's Arnoldi;
* T_m = S_m^H A S_m is triangular only up to the residual of the
  eigenvectors; its strictly lower part is dropped (the paper stores the
  triangular matrix);
* S_m comes from a QR factorisation of R_m in the given column order, so
  that its leading columns span the leading eigenvectors;
* App. A prints the upper limit of the sums over H as max(j+1, n); H is
  upper Hessenberg, so column j has entries in rows 1..j+1 only and the
  limit is min(j+1, n).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""

import numpy as np

from .newton import roberts_sign
from .arnoldi import BREAKDOWN_TOL


def schur_from_eigvecs(matvec_block, r):
    """S_m (orthonormal, N x m) and upper triangular T_m from right
    eigenvectors r (N x m) of A (Sec. 5.2 step i). ``matvec_block(S)``
    returns A S."""
    s, _ = np.linalg.qr(np.asarray(r, dtype=np.complex128))
    t = s.conj().T @ matvec_block(s)
    return s, np.triu(t)


def sylvester_rowwise(t, h, c):
    """Solve T Y - Y H = C for Y (App. A): T (m x m) upper triangular, H
    (n x n) upper Hessenberg with nonzero subdiagonal, C (m x n).

    Rows are solved from the bottom up (Eq. SolveRow with the known rows
    below folded into c~). Inside row i every element is y_ij = a_j y_i1 +
    b_j (Eq. xij) with a_1 = 1, b_1 = 0 and the recurrences of Eq. abij
    (Eq. SolveComp); y_i1 then follows from element (i, n) of Eq. SolveRow.
    Indices below are 0-based: paper column j is index j - 1.
    """
    t = np.asarray(t, dtype=np.complex128)
    h = np.asarray(h, dtype=np.complex128)
    c = np.asarray(c, dtype=np.complex128)
    m, n = c.shape
    y = np.zeros((m, n), dtype=np.complex128)
    for i in range(m - 1, -1, -1):
        # c~_ij = c_ij - sum_{k > i} T_ik y_kj
        ct = c[i] - t[i, i + 1:] @ y[i + 1:]
        tii = t[i, i]
        a = np.zeros(n, dtype=np.complex128)
        b = np.zeros(n, dtype=np.complex128)
        a[0] = 1.0
        for j in range(n - 1):
            # sums over k = 1 .. min(j+1, n) (paper indices) of column j:
            # 0-based rows 0 .. j (row j+1 is the subdiagonal, solved for)
            sa = a[: j + 1] @ h[: j + 1, j]
            sb = b[: j + 1] @ h[: j + 1, j]
            a[j + 1] = -(-tii * a[j] + sa) / h[j + 1, j]
            b[j + 1] = -(ct[j] - tii * b[j] + sb) / h[j + 1, j]
        # element (i, n): T_ii y_in - sum_k y_ik H_kn = c~_in
        num = ct[n - 1] - tii * b[n - 1] + b @ h[:, n - 1]
        den = tii * a[n - 1] - a @ h[:, n - 1]
        y[i] = a * (num / den) + b
    return y


def modified_arnoldi(matvec, x_perp, s, k):
    """Arnoldi on x_perp with every vector orthogonalised against the Schur
    vectors s and the previous Arnoldi vectors (Eq. modArnoldi), classical
    Gram-Schmidt applied twice.

    Returns (V, H, X, beta, k_used): V is N x (k_used+1), H (k_used+1) x
    k_used upper Hessenberg, X = S^H A V_(k_used) (m x k_used).
    """
    x_perp = np.asarray(x_perp, dtype=np.complex128)
    n = x_perp.shape[0]
    m = s.shape[1]
    beta = np.linalg.norm(x_perp)
    v = np.zeros((n, k + 1), dtype=np.complex128)
    hh = np.zeros((k + 1, k), dtype=np.complex128)
    xx = np.zeros((m, k), dtype=np.complex128)
    if beta == 0.0 or k == 0:
        return v[:, :1], hh[:1, :0], xx[:, :0], beta, 0
    v[:, 0] = x_perp / beta
    for j in range(k):
        w = matvec(v[:, j])
        q = np.hstack([s, v[:, : j + 1]])
        h1 = q.conj().T @ w
        w = w - q @ h1
        h2 = q.conj().T @ w
        w = w - q @ h2
        col = h1 + h2
        xx[:, j] = col[:m]
        hh[: j + 1, j] = col[m:]
        hn = np.linalg.norm(w)
        hh[j + 1, j] = hn
        if hn <= BREAKDOWN_TOL * np.linalg.norm(hh[: j + 2, : j + 1]):
            hh[j + 1, j] = 0.0
            return v[:, : j + 2] * np.r_[np.ones(j + 1), 0.0], hh[: j + 2, : j + 1], xx[:, : j + 1], beta, j + 1
        v[:, j + 1] = w / hn
    return v, hh, xx, beta, k


def schur_sign_apply(matvec, x, s, t, k, f_t=None, **newton_kw):
    """sgn(A) x by Schur deflation (Sec. 5.2 steps iii-vi, Eq. formula).

    ``s``: N x m orthonormal Schur vectors, ``t``: m x m upper triangular
    with A S = S T, ``f_t``: sgn(T) (computed by Roberts' iteration if not
    given). Returns (y, info) with info = dict(k_used, beta, newton_iters,
    c (= S^H x), coeff_s (the S coefficients), coeff_v, Y, X, H).
    """
    x = np.asarray(x, dtype=np.complex128)
    if f_t is None:
        f_t, _ = roberts_sign(t, **newton_kw)
    c = s.conj().T @ x
    x_perp = x - s @ c
    v, hh, xx, beta, k_used = modified_arnoldi(matvec, x_perp, s, k)
    y_s = f_t @ c
    if k_used == 0:
        return s @ y_s, dict(k_used=0, beta=beta, newton_iters=0, c=c, coeff_s=y_s,
                             coeff_v=np.zeros(0, np.complex128))
    hk = hh[:k_used, :k_used]
    f_h, it = roberts_sign(hk, **newton_kw)
    # App. A divides by the subdiagonal of H_k, which is nonzero for every
    # step the Arnoldi recurrence kept (a breakdown ends H_k before a zero)
    cc = f_t @ xx - xx @ f_h
    yy = sylvester_rowwise(t, hk, cc)
    coeff_s = y_s + beta * yy[:, 0]
    coeff_v = beta * f_h[:, 0]
    y = s @ coeff_s + v[:, :k_used] @ coeff_v
    return y, dict(k_used=k_used, beta=beta, newton_iters=it, c=c, coeff_s=coeff_s, coeff_v=coeff_v,
                   Y=yy, X=xx, H=hh)
