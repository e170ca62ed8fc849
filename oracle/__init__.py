"""CPU oracle for sgn(H_w(mu)) x (Bloch, Frommer, Lang, Wettig 2007).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product path
(the CUDA library and its Python binding) never imports, links or calls it,
and this package never imports the product.

Plain, slow and written to be checked against the paper by eye: numpy/scipy
in complex128, no blocking or fusion beyond what each formula states.

Modules and the passages they follow:

* ``lattice``   -- gamma matrices, D_w(mu) and H_w(mu) = gamma5 D_w(mu) as a
                   sparse matrix built term by term, and the same sum
                   evaluated at chosen sites only for large lattices
                   (Sec. 2, Eq. Dw).
* ``signfun``   -- complex sign (Sec. 2, Eq. sgnz) and the spectral matrix
                   function f(A) = U f(Lambda) U^-1 (Sec. 2, Eq. fA).
* ``newton``    -- Roberts' iteration S <- (S + S^-1)/2 (Sec. 5.2, Eq. Roberts).
* ``arnoldi``   -- Arnoldi recurrence with classical Gram-Schmidt applied
                   twice (Sec. 4, Eqs. Arnoldi, HVAV) and the approximation
                   f(A)x ~ beta V_k f(H_k) e_1 (Sec. 4, Eq. yproj3), at a
                   fixed k or stopped by the change of the coefficient
                   vector between checks (the batched form's criterion),
                   the checks every interval or on the skip-ahead schedule.
* ``deflation`` -- LR deflation (Sec. 5.3, Eqs. Rev, Lev, xdec, fAxLR, fARLx,
                   LRArnoldi, fAxLRArn), also with the adaptive stop, and
                   critical eigenpairs (Sec. 6).
* ``schur``     -- Schur deflation (Sec. 5.2, Eqs. pSd, modArnoldi, newH,
                   f_H, SylvEq, formula) with the row-by-row Sylvester
                   solver of App. A (Eqs. GenSylvEq to abij).
* ``overlap``   -- D_ov(mu) = 1 + gamma5 sgn(H_w(mu)) (Sec. 2, Eqs. Dov,
                   GW:eq) and restarted GMRES for the nested inversion the
                   paper names as the method's use (Secs. 6, 7).
* ``freefield`` -- unit-link (free) closed form of D_w, H_w and sgn(H_w) in
                   momentum space; an independent pin for the above.

``arnoldi`` also holds the harmonic (see-saw-free) variant of Sec. 4.

Pins (tests marked ``not gpu``): the free-field closed form, gauge
covariance, gamma5-hermiticity, the Hermitian mu = 0 case (sgn equals the
polar factor), sgn(A)^2 = I, Arnoldi exactness at the grade of x, Newton
against scipy.linalg.signm and against matrices of known eigen-decomposition,
LR deflation on exact eigenvectors, the per-site sum against the pure-gauge
closed form, the adaptive stop against the fixed-k form and the dense sign,
the ARPACK critical pairs against the dense spectral projector, the App. A
solver against scipy's Sylvester solver and the spectral sign of the
composite matrix, harmonic Ritz values against their Petrov-Galerkin
definition, the Ginsparg-Wilson relation and GMRES against a dense solve.
Parity pinned for every function.
"""

from . import lattice, signfun, newton, arnoldi, deflation, freefield, schur, overlap  # noqa: F401
