"""Seeded source vectors (canonical layout [nrhs][N], N = 12 V)."""

import numpy as np


def gaussian_vectors(n, nrhs, seed):
    """nrhs complex Gaussian vectors of length n, each of unit 2-norm.

    Real and imaginary parts are iid N(0, 1) from numpy's PCG64 seeded with
    ``seed``; the vectors are then scaled to unit norm.
    """
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    x = rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x


def ones_vector(n):
    """The source x = (1, ..., 1) used for the paper's convergence figures."""
    return np.ones((1, n), dtype=np.complex128)


def plane_wave_vectors(dims, modes, seed, omega=None):
    """Sum of a few plane waves, antiperiodic in t.

    ``modes`` is a list of integer 4-tuples (kx, ky, kz, kt); mode k carries
    momentum p_nu = 2 pi k_nu / L_nu (nu < 3) and p_t = 2 pi (k_t + 1/2) / L_t.
    Each mode gets a random (seeded) 12-component spin-colour amplitude.
    If ``omega`` ([V][3][3]) is given, the colour index is rotated by
    omega(s), so the vector matches a pure-gauge field built from omega.
    Returns a [1][N] complex128 array of unit norm.
    """
    lx, ly, lz, lt = (int(d) for d in dims)
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    field = np.zeros((lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    for (kx, ky, kz, kt) in modes:
        amp = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        phase = np.exp(1j * (2 * np.pi * kx * x / lx + 2 * np.pi * ky * y / ly
                             + 2 * np.pi * kz * z / lz + 2 * np.pi * (kt + 0.5) * t / lt))
        field += phase[..., None, None] * amp
    field = field.reshape(-1, 4, 3)
    if omega is not None:
        field = np.einsum("sab,sib->sia", omega, field)
    out = field.reshape(1, -1)
    return out / np.linalg.norm(out)
