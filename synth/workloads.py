"""Seeded instance recipe of the batched multi-instance workload.

Instance i (i = 0, 1, ...): lattice cycling through 4^4, 6^4, 8^4; mu cycling
through 0.1, 0.2, 0.3; gauge roughness eps uniform in [0.5, 0.7] drawn from
numpy's PCG64 with seed 100 + i, and the gauge field itself from seed 100 + i;
right-hand-side count 1 + (h(i) mod 16), h the splitmix64 finaliser (an
integer mixing function, so the counts are spread unevenly); sources from
seed 200 + i. m_w = -1.5 throughout.
"""

import numpy as np

_MASK = (1 << 64) - 1


def _splitmix64(i):
    z = (i + 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def batched_instances(n):
    """List of n dicts: dims, gauge_seed, eps, mu, nrhs, source_seed."""
    sizes = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 8)]
    out = []
    for i in range(n):
        eps = float(np.random.default_rng(100 + i).uniform(0.5, 0.7))
        out.append({"dims": sizes[i % 3], "gauge_seed": 100 + i, "eps": eps, "mu": (0.1, 0.2, 0.3)[i % 3],
                    "nrhs": 1 + int(_splitmix64(i) % 16), "source_seed": 200 + i})
    return out


def synthetic_deflation(n, m, seed):
    """Seeded stand-in deflation data: R, L (n x m complex Gaussian) and
    lambda with |Re lambda| uniform in [0.05, 0.5], random sign, and
    Im lambda uniform in [-0.3, 0.3]. Not eigenpairs of any operator: the LR
    formula is defined for any biorthonormalisable (R, L)."""
    from .vectors import gaussian_vectors
    r = gaussian_vectors(n, m, seed).T.copy()
    l = gaussian_vectors(n, m, seed + 1).T.copy()
    rng = np.random.default_rng(seed)
    lam = rng.uniform(0.05, 0.5, m) * rng.choice([-1.0, 1.0], m) + 1j * rng.uniform(-0.3, 0.3, m)
    return r, l, lam
