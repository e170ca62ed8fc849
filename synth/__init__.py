"""Seeded synthetic inputs shared by the CUDA path's tests and the oracle.

This module holds no arithmetic of the sign-function method. It only makes
inputs: SU(3) gauge links U = exp(i eps X) and complex Gaussian source vectors,
with the shapes and distributions of the workloads the method is run on (the
paper's beta_g = 5.1 gauge ensembles are not available; a seeded near-identity
random SU(3) field stands in for them).

Conventions (also those of the C library):

* lattice dims (Lx, Ly, Lz, Lt); site s = ((t*Lz + z)*Ly + y)*Lx + x;
* direction nu = 0, 1, 2, 3 for x, y, z, t (the paper's nu = 1..4);
* links: complex128 array [V][4][3][3] (row, column), U_nu(s) joins s to s+nu;
* vectors: complex128 [nrhs][N], N = 12 V, index (s*4 + spin)*3 + colour.

The gauge generator is counter based (Philox4x32-10, Salmon et al., SC'11,
"Parallel random numbers: as easy as 1, 2, 3") so that the C library's
``ovs_create_gauge`` can produce the same field from the same seed without
sharing code with this module.
"""

from .philox import philox4x32_10, philox_uniform52
from .gauge import gauge_links, unit_links, pure_gauge_links, random_su3, link_count
from .vectors import gaussian_vectors, ones_vector, plane_wave_vectors
from .workloads import batched_instances, synthetic_deflation

__all__ = [
    "philox4x32_10",
    "philox_uniform52",
    "gauge_links",
    "unit_links",
    "pure_gauge_links",
    "random_su3",
    "link_count",
    "gaussian_vectors",
    "ones_vector",
    "plane_wave_vectors",
    "batched_instances",
    "synthetic_deflation",
]
