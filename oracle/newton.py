"""Roberts' Newton iteration for the matrix sign (Sec. 5.2, Eq. Roberts).

S^0 = A,  S^(n+1) = (S^n + (S^n)^-1) / 2, which converges quadratically to
sgn(A) when no eigenvalue of A lies on the imaginary axis. The paper applies
it to the Hessenberg matrix H_k (Sec. 5.3, step v) and keeps the first
column.

Stopping rule (the paper gives none): stop after the first iterate whose
relative change ||S^(n+1) - S^n||_F / ||S^(n+1)||_F is <= ``switch_tol``
plus ``extra`` more iterations (quadratic convergence makes one extra
iteration reach rounding level), or fail after ``max_iter`` iterations.
"""

import numpy as np


class NewtonNotConverged(RuntimeError):
    pass


def roberts_sign(a, switch_tol=1e-9, extra=1, max_iter=50):
    """Return (sgn(A), iterations) by S <- (S + S^-1)/2 with S^0 = A."""
    s = np.array(a, dtype=np.complex128, copy=True)
    if s.shape[0] == 0:
        return s, 0
    remaining = None
    for it in range(1, max_iter + 1):
        s_new = 0.5 * (s + np.linalg.inv(s))
        change = np.linalg.norm(s_new - s) / np.linalg.norm(s_new)
        s = s_new
        if remaining is None and change <= switch_tol:
            remaining = extra
        if remaining is not None:
            if remaining == 0:
                return s, it
            remaining -= 1
    raise NewtonNotConverged(f"Roberts iteration did not converge in {max_iter} steps")


def sign_first_column(h, beta, **kw):
    """beta * sgn(H) e_1, the coefficient vector of Eq. yproj3."""
    s, it = roberts_sign(h, **kw)
    return beta * s[:, 0], it
