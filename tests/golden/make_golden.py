"""Writes the stored expected values under tests/golden/ from the oracle
alone (run from the repository root: python tests/golden/make_golden.py).

freefield_2x2x2x4.txt: the spectrum of the free (unit-link) H_w(mu) =
gamma5 D_w(mu) (Sec. 2, Eqs. Dov and Dw) on a 2x2x2x4 lattice, antiperiodic
in time, m_w = -1.5, at mu = 0 and mu = 0.3, from the momentum-space closed
form of oracle.freefield: one line per momentum and sign (each value is
6-fold there: 2 spins x 3 colours), sorted by (Re, Im).
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import freefield  # noqa: E402

DIMS, MW = (2, 2, 2, 4), -1.5


def main():
    lines = ["# spectrum of the free H_w(mu) (Sec. 2, Eqs. Dov, Dw), 2x2x2x4, antiperiodic in time, m_w = -1.5",
             "# each eigenvalue 6-fold (2 spins x 3 colours); written by tests/golden/make_golden.py (oracle.freefield)",
             "# mu re im"]
    for mu in (0.0, 0.3):
        z = freefield.spectrum(DIMS, mu, MW)
        z = z[np.lexsort((np.round(z.imag, 12), np.round(z.real, 12)))]
        for v in z:
            lines.append(f"{mu:.1f} {v.real:.17e} {v.imag:.17e}")
    with open(os.path.join(HERE, "freefield_2x2x2x4.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
