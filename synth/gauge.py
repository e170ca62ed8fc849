"""Seeded SU(3) gauge links U = exp(i eps X) (input recipe of the workloads).

Recipe, per link l = 4*s + nu, key (seed mod 2**32, seed div 2**32):

1. nine Philox4x32-10 calls with counter (l mod 2**32, l div 2**32, j, 0),
   j = 0..8; call j gives uniforms u0 = U52(w0, w1), u1 = U52(w2, w3) and the
   Box-Muller pair r cos(2 pi u1), r sin(2 pi u1), r = sqrt(-2 ln u0), which
   are entries 2j and 2j+1 of eighteen normals n;
2. A[a][b] = n[2(3a+b)] + i n[2(3a+b)+1];
3. X = (A + A^dagger)/2 minus (tr/3) times the identity (traceless Hermitian);
4. U = exp(i eps X) by scaling and squaring: s = least s >= 0 with
   ||i eps X||_F / 2**s <= 1/2, Taylor series of degree 18, squared s times;
5. reunitarise: normalise row 0, Gram-Schmidt row 1 against it and normalise,
   row 2 = complex conjugate of (row 0 x row 1), so det U = 1.
"""

import numpy as np

from .philox import philox4x32_10, philox_uniform52

_TAYLOR_DEGREE = 18
_TWO_PI = 6.283185307179586


def link_count(dims):
    lx, ly, lz, lt = (int(d) for d in dims)
    return lx * ly * lz * lt * 4


def _normals18(index, seed):
    """Eighteen standard normals per counter index (array of int64)."""
    index = np.asarray(index, dtype=np.uint64)
    lo = index & np.uint64(0xFFFFFFFF)
    hi = index >> np.uint64(32)
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    out = np.empty(index.shape + (18,), dtype=np.float64)
    for j in range(9):
        w0, w1, w2, w3 = philox4x32_10(lo, hi, np.uint64(j), np.uint64(0), k0, k1)
        u0 = philox_uniform52(w0, w1)
        u1 = philox_uniform52(w2, w3)
        r = np.sqrt(-2.0 * np.log(u0))
        out[..., 2 * j] = r * np.cos(_TWO_PI * u1)
        out[..., 2 * j + 1] = r * np.sin(_TWO_PI * u1)
    return out


def _expm_taylor(m):
    """exp of a stack of 3x3 complex matrices by scaling and squaring."""
    nrm = np.sqrt(np.sum(np.abs(m) ** 2, axis=(-2, -1)))
    s = np.zeros(nrm.shape, dtype=np.int64)
    big = nrm > 0.5
    s[big] = np.ceil(np.log2(nrm[big] / 0.5)).astype(np.int64)
    # guard against log2 rounding: make sure the scaled norm is <= 1/2
    while True:
        over = nrm / np.ldexp(1.0, s) > 0.5
        if not np.any(over):
            break
        s[over] += 1
    ms = m / np.ldexp(1.0, s)[..., None, None]
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), m.shape)
    result = eye.copy()
    term = eye.copy()
    for n in range(1, _TAYLOR_DEGREE + 1):
        term = np.matmul(term, ms) / n
        result = result + term
    smax = int(s.max()) if s.size else 0
    for it in range(smax):
        sel = s > it
        result[sel] = np.matmul(result[sel], result[sel])
    return result


def _reunitarise(u):
    r0 = u[..., 0, :]
    r1 = u[..., 1, :]
    r0 = r0 / np.sqrt(np.sum(np.abs(r0) ** 2, axis=-1))[..., None]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1)[..., None] * r0
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1))[..., None]
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def random_su3(index, seed, eps):
    """SU(3) matrices exp(i eps X) for an array of counter indices."""
    n = _normals18(index, seed)
    a = (n[..., 0::2] + 1j * n[..., 1::2]).reshape(n.shape[:-1] + (3, 3))
    x = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(x, axis1=-2, axis2=-1) / 3.0
    x = x - tr[..., None, None] * np.eye(3)
    return _reunitarise(_expm_taylor(1j * eps * x))


def gauge_links(dims, seed, eps):
    """Links [V][4][3][3] complex128 for lattice dims (Lx, Ly, Lz, Lt)."""
    nl = link_count(dims)
    u = random_su3(np.arange(nl, dtype=np.int64), int(seed), float(eps))
    return u.reshape(nl // 4, 4, 3, 3)


def unit_links(dims):
    """The free field: every link is the identity."""
    v = link_count(dims) // 4
    u = np.zeros((v, 4, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def _site_shift(dims, nu, step):
    lx, ly, lz, lt = dims
    s = np.arange(lx * ly * lz * lt)
    c = [s % lx, (s // lx) % ly, (s // (lx * ly)) % lz, s // (lx * ly * lz)]
    c[nu] = (c[nu] + step) % dims[nu]
    return ((c[3] * lz + c[2]) * ly + c[1]) * lx + c[0]


def pure_gauge_links(dims, seed):
    """Pure-gauge field U_nu(s) = Omega(s) Omega(s+nu)^dagger.

    Returns (links, omega) with omega [V][3][3] generic SU(3) (eps = 3).
    """
    dims = tuple(int(d) for d in dims)
    v = dims[0] * dims[1] * dims[2] * dims[3]
    omega = random_su3(np.arange(v, dtype=np.int64), int(seed), 3.0)
    u = np.empty((v, 4, 3, 3), dtype=np.complex128)
    for nu in range(4):
        fwd = _site_shift(dims, nu, +1)
        u[:, nu] = np.matmul(omega, np.conj(np.swapaxes(omega[fwd], -1, -2)))
    return u, omega
