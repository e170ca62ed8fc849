"""Complex and matrix sign by the spectral definition.

* sgn(z) = z / sqrt(z^2) = sgn(Re z), principal square root with the cut on
  the negative real axis (Sec. 2, Eq. sgnz);
* f(A) = U f(Lambda) U^-1 for diagonalisable A (Sec. 2, Eq. fA), hence
  sgn(A) = U diag(sgn(Re lambda_i)) U^-1 (Sec. 2, Eq. signA).

The paper assumes diagonalisable matrices in practice (Sec. 5.1, end).
"""

import numpy as np


def sgn_scalar(z):
    """sgn(z) = z / sqrt(z^2); equals sgn(Re z) away from the imaginary axis."""
    z = np.asarray(z, dtype=np.complex128)
    return z / np.sqrt(z * z)


def sgn_re(z):
    """sgn(Re z) as +1/-1 (real). Raises on Re z == 0, where it is undefined."""
    re = np.real(np.asarray(z))
    if np.any(re == 0):
        raise ValueError("sign undefined on the imaginary axis")
    return np.where(re > 0, 1.0, -1.0)


def eig_decomposition(a):
    """Dense eigen-decomposition A = U diag(lam) U^-1 (LAPACK geev)."""
    lam, u = np.linalg.eig(np.asarray(a, dtype=np.complex128))
    return lam, u


def sgn_matrix(a):
    """Full sign matrix U diag(sgn(Re lam)) U^-1 (Eq. fA with Eq. sgnz)."""
    lam, u = eig_decomposition(a)
    return u @ np.diag(sgn_re(lam)) @ np.linalg.inv(u)


def sgn_apply_dense(a, x, decomposition=None):
    """y = sgn(A) x by the spectral definition; x may be [N] or [N][nrhs]."""
    if decomposition is None:
        decomposition = eig_decomposition(a)
    lam, u = decomposition
    coeff = np.linalg.solve(u, x)
    s = sgn_re(lam)
    if coeff.ndim == 1:
        return u @ (s * coeff)
    return u @ (s[:, None] * coeff)


def polar_factor(a):
    """pol(A) = A (A^dagger A)^(-1/2) via the SVD A = W S Z^dagger -> W Z^dagger."""
    w, _, zh = np.linalg.svd(np.asarray(a, dtype=np.complex128))
    return w @ zh
