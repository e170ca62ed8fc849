"""Wilson-Dirac operator at chemical potential, written term by term.

Follows Sec. 2, Eq. Dw: D_w(mu) is the identity minus kappa times eight
nearest-neighbour hops, each a spin projector (1 -/+ gamma_nu) times an SU(3)
link, the temporal hops weighted by exp(+mu) (forward) and exp(-mu)
(backward); kappa = 1/(8 + 2 m_w). H_w(mu) = gamma5 D_w(mu) (Sec. 2, Eq. Dov).

Readings where the paper is silent:

* gamma matrices: chiral basis, gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]
  (k = 1, 2, 3), gamma_4 = [[0, 1], [1, 0]], so gamma5 = gamma1 gamma2 gamma3
  gamma4 = diag(1, 1, -1, -1);
* boundary conditions: periodic in space, antiperiodic in time (a factor -1
  on every hop that wraps around in t);
* hop convention: the default ``"minus_forward"`` puts (1 - gamma_nu) on the
  forward hop and (1 + gamma_nu) on the backward hop; ``"paper"`` is Eq. Dw as
  printed, (1 + gamma_j) forward and (1 - gamma_j) backward. The two are
  related by D_paper = gamma5 D_minus_forward gamma5, so they share the spectrum
  and sgn(H_paper) = gamma5 sgn(H_minus_forward) gamma5.

Index of a vector entry: (s*4 + spin)*3 + colour, s = ((t*Lz+z)*Ly+y)*Lx+x.
"""

import numpy as np
import scipy.sparse as sp

_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def gamma_matrices():
    """gamma_1..gamma_4 (Euclidean, Hermitian) in the chiral basis."""
    g = [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in SIGMA]
    g.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
    return g


def gamma5():
    g = gamma_matrices()
    return g[0] @ g[1] @ g[2] @ g[3]


def kappa_of(m_w):
    """kappa = 1/(8 + 2 m_w) (Sec. 2, after Eq. Dw)."""
    return 1.0 / (8.0 + 2.0 * m_w)


def site_coords(dims):
    lx, ly, lz, lt = dims
    s = np.arange(lx * ly * lz * lt)
    return [s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)]


def neighbour(dims, nu, step):
    """Site index of s + step*nu-hat (periodic wrap) and the wrap flag."""
    lx, ly, lz, lt = dims
    c = site_coords(dims)
    raw = c[nu] + step
    wrapped = (raw < 0) | (raw >= dims[nu])
    c[nu] = raw % dims[nu]
    return ((c[3] * lz + c[2]) * ly + c[1]) * lx + c[0], wrapped


def _hop_blocks(spin, links):
    """12x12 blocks kron(spin, link) per site; rows (a, c), columns (b, d)."""
    v = links.shape[0]
    blk = np.einsum("ab,scd->sacbd", spin, links)
    return blk.reshape(v, 12, 12)


def wilson_dirac(links, dims, mu, m_w, convention="minus_forward"):
    """Sparse D_w(mu) (N x N, N = 12 V) built hop by hop from Eq. Dw."""
    dims = tuple(int(d) for d in dims)
    v = dims[0] * dims[1] * dims[2] * dims[3]
    n = 12 * v
    kappa = kappa_of(m_w)
    gam = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    sign_fwd = -1.0 if convention == "minus_forward" else +1.0
    if convention not in ("minus_forward", "paper"):
        raise ValueError("convention must be 'minus_forward' or 'paper'")
    sites = np.arange(v)
    rows_all, cols_all, vals_all = [], [], []
    # diagonal delta_{n,m}
    rows_all.append(np.arange(n))
    cols_all.append(np.arange(n))
    vals_all.append(np.ones(n, dtype=np.complex128))
    idx = np.arange(12)
    for nu in range(4):
        tfac = np.exp(mu) if nu == 3 else 1.0
        # forward hop: psi(s + nu) through U_nu(s)
        fwd, wrap_f = neighbour(dims, nu, +1)
        bc_f = np.where(wrap_f & (nu == 3), -1.0, 1.0)
        p_fwd = one + sign_fwd * gam[nu]
        blk = _hop_blocks(p_fwd, links[:, nu])
        blk = blk * (-kappa * tfac * bc_f)[:, None, None]
        rows_all.append(np.repeat(12 * sites[:, None] + idx[None, :], 12, axis=1).ravel())
        cols_all.append(np.tile(12 * fwd[:, None] + idx[None, :], (1, 12)).ravel())
        vals_all.append(blk.ravel())
        # backward hop: psi(s - nu) through U_nu(s - nu)^dagger
        bwd, wrap_b = neighbour(dims, nu, -1)
        bc_b = np.where(wrap_b & (nu == 3), -1.0, 1.0)
        p_bwd = one - sign_fwd * gam[nu]
        udag = np.conj(np.swapaxes(links[bwd, nu], -1, -2))
        blk = _hop_blocks(p_bwd, udag)
        blk = blk * (-kappa / tfac * bc_b)[:, None, None]
        rows_all.append(np.repeat(12 * sites[:, None] + idx[None, :], 12, axis=1).ravel())
        cols_all.append(np.tile(12 * bwd[:, None] + idx[None, :], (1, 12)).ravel())
        vals_all.append(blk.ravel())
    rows = np.concatenate(rows_all)
    cols = np.concatenate(cols_all)
    vals = np.concatenate(vals_all)
    keep = vals != 0
    d = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n, n)).tocsr()
    d.sum_duplicates()
    return d


def wilson_dirac_sites(links, dims, mu, m_w, x, sites, convention="minus_forward"):
    """(D_w(mu) x) at the listed sites only, as an array (len(sites), 12).

    Each of the eight hops of Eq. Dw is summed directly for the requested
    sites, without forming the matrix, so that lattices too large for the
    sparse form (16^3 x 32: N = 1.57 M) can still be checked site by site.
    Same readings as ``wilson_dirac``.
    """
    dims = tuple(int(d) for d in dims)
    lx, ly, lz, lt = dims
    sites = np.asarray(sites, dtype=np.int64)
    if convention not in ("minus_forward", "paper"):
        raise ValueError("convention must be 'minus_forward' or 'paper'")
    sign_fwd = -1.0 if convention == "minus_forward" else +1.0
    kappa = kappa_of(m_w)
    gam = gamma_matrices()
    one = np.eye(4, dtype=np.complex128)
    psi = np.asarray(x, dtype=np.complex128).reshape(-1, 4, 3)
    coord = [sites % lx, (sites // lx) % ly, (sites // (lx * ly)) % lz, sites // (lx * ly * lz)]
    out = psi[sites].copy()
    for nu in range(4):
        tfac = np.exp(mu) if nu == 3 else 1.0
        for step in (+1, -1):
            c = [a.copy() for a in coord]
            raw = coord[nu] + step
            wrapped = (raw < 0) | (raw >= dims[nu])
            c[nu] = raw % dims[nu]
            nb = ((c[3] * lz + c[2]) * ly + c[1]) * lx + c[0]
            bc = np.where(wrapped & (nu == 3), -1.0, 1.0)
            if step > 0:  # psi(s + nu) through U_nu(s), (1 - gamma_nu) in the minus_forward convention
                proj = one + sign_fwd * gam[nu]
                u = links[sites, nu]
                w = tfac
            else:  # psi(s - nu) through U_nu(s - nu)^dagger
                proj = one - sign_fwd * gam[nu]
                u = np.conj(np.swapaxes(links[nb, nu], -1, -2))
                w = 1.0 / tfac
            term = np.einsum("ab,scd,sbd->sac", proj, u, psi[nb])
            out -= (kappa * w * bc)[:, None, None] * term
    return out.reshape(len(sites), 12)


def hw_sites(links, dims, mu, m_w, x, sites, convention="minus_forward"):
    """(H_w(mu) x) = (gamma5 D_w(mu) x) at the listed sites (Sec. 2, Eq. Dov)."""
    d = wilson_dirac_sites(links, dims, mu, m_w, x, sites, convention)
    return d * np.repeat(np.real(np.diag(gamma5())), 3)[None, :]


def gamma5_diag(v):
    """Diagonal of gamma5 (x) 1_colour over all sites, length 12 V."""
    g5 = np.real(np.diag(gamma5()))
    return np.tile(np.repeat(g5, 3), v)


def hw_operator(links, dims, mu, m_w, convention="minus_forward"):
    """Sparse H_w(mu) = gamma5 D_w(mu) (Sec. 2, Eq. Dov)."""
    d = wilson_dirac(links, dims, mu, m_w, convention)
    v = d.shape[0] // 12
    return sp.diags(gamma5_diag(v)) @ d
