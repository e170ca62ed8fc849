"""Free-field (unit link) closed form of D_w(mu), H_w(mu) and sgn(H_w(mu)).

With every link equal to the identity, Eq. Dw is diagonal in momentum space.
For a plane wave e^{i p.n} (p_nu = 2 pi k_nu / L_nu in space and
p_4 = 2 pi (k_4 + 1/2) / L_t for the antiperiodic time direction), set
p~_nu = p_nu for nu < 4 and p~_4 = p_4 - i mu. The forward hop contributes
(1 - gamma_nu) e^{i p~_nu} and the backward hop (1 + gamma_nu) e^{-i p~_nu}
(hop convention "minus_forward"), so

    D(p) = a + i sum_nu b_nu gamma_nu,
    a    = 1 - 2 kappa sum_nu cos p~_nu,   b_nu = 2 kappa sin p~_nu,

and, since gamma5 gamma_nu gamma5 = -gamma_nu and {gamma_mu, gamma_nu} = 2
delta, H(p)^2 = (gamma5 D(p))^2 = (a^2 + b.b) 1. Every eigenvalue z of H(p)
has z^2 = a^2 + b.b, so by Eq. sgnz, sgn(H(p)) = H(p) / sqrt(a^2 + b.b) with
the principal square root.

A pure-gauge field U_nu(n) = Omega(n) Omega(n+nu)^dagger gives
D[U] = Omega D[1] Omega^dagger (gauge covariance), so the same formulas hold
after rotating the colour index by Omega.
"""

import numpy as np

from .lattice import gamma_matrices, gamma5, kappa_of


def _momentum_grid(dims):
    lx, ly, lz, lt = dims
    kt, kz, ky, kx = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    px = 2 * np.pi * kx / lx
    py = 2 * np.pi * ky / ly
    pz = 2 * np.pi * kz / lz
    pt = 2 * np.pi * (kt + 0.5) / lt
    return [px, py, pz, pt]


def symbol(dims, mu, m_w):
    """Return (a, b) on the momentum grid (axes t, z, y, x); b has 4 entries."""
    kappa = kappa_of(m_w)
    p = _momentum_grid(tuple(int(d) for d in dims))
    pt = [p[0], p[1], p[2], p[3] - 1j * mu]
    a = 1.0 - 2.0 * kappa * sum(np.cos(q) for q in pt)
    b = [2.0 * kappa * np.sin(q) for q in pt]
    return a, b


def _spin_matrix_field(dims, mu, m_w, kind):
    a, b = symbol(dims, mu, m_w)
    g = gamma_matrices()
    g5 = gamma5()
    d = a[..., None, None] * np.eye(4) + 1j * sum(b[n][..., None, None] * g[n] for n in range(4))
    if kind == "D":
        return d
    h = np.einsum("ab,...bc->...ac", g5, d)
    if kind == "H":
        return h
    if kind == "sgnH":
        delta = a * a + sum(bn * bn for bn in b)
        return h / np.sqrt(delta)[..., None, None]
    raise ValueError(kind)


def apply_free(x, dims, mu, m_w, kind="sgnH", omega=None):
    """Apply D, H or sgn(H) of the free (or pure-gauge) field to x [N]."""
    lx, ly, lz, lt = (int(d) for d in dims)
    dims = (lx, ly, lz, lt)
    f = np.asarray(x, dtype=np.complex128).reshape(lt * lz * ly * lx, 4, 3)
    if omega is not None:
        f = np.einsum("sba,sib->sia", np.conj(omega), f)  # Omega^dagger x
    f = f.reshape(lt, lz, ly, lx, 4, 3)
    tw = np.exp(1j * np.pi * np.arange(lt) / lt)[:, None, None, None, None, None]
    fk = np.fft.fftn(f / tw, axes=(0, 1, 2, 3))
    m = _spin_matrix_field(dims, mu, m_w, kind)
    gk = np.einsum("...ab,...bc->...ac", m, fk)
    g = np.fft.ifftn(gk, axes=(0, 1, 2, 3)) * tw
    g = g.reshape(-1, 4, 3)
    if omega is not None:
        g = np.einsum("sab,sib->sia", omega, g)
    return g.reshape(-1)


def spectrum(dims, mu, m_w):
    """All eigenvalues of the free H_w(mu): +/- sqrt(a^2 + b.b), each 6-fold
    (2 spin x 3 colour); returned once per momentum and sign."""
    a, b = symbol(dims, mu, m_w)
    root = np.sqrt(a * a + sum(bn * bn for bn in b)).ravel()
    return np.concatenate([root, -root])
