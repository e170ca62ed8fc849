"""Stored expected values (tests/golden/, written from the oracle by
tests/golden/make_golden.py): the spectrum of the free H_w(mu) on a
2x2x2x4 lattice from the momentum-space closed form. The term-by-term
sparse operator of oracle.lattice, an independent construction of Eq. Dw,
must have exactly these eigenvalues, each 6-fold; the closed form must
still produce them."""

import os

import numpy as np

import synth
from oracle import freefield, lattice

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
DIMS, MW = (2, 2, 2, 4), -1.5


def _stored():
    rows = np.loadtxt(os.path.join(HERE, "freefield_2x2x2x4.txt"), comments="#")
    return {mu: rows[rows[:, 0] == mu][:, 1] + 1j * rows[rows[:, 0] == mu][:, 2] for mu in np.unique(rows[:, 0])}


def _sorted(z):
    return z[np.lexsort((np.round(z.imag, 9), np.round(z.real, 9)))]


def test_free_spectrum_of_the_lattice_operator_matches_stored():
    stored = _stored()
    assert sorted(stored) == [0.0, 0.3]
    for mu, z in stored.items():
        h = lattice.hw_operator(synth.unit_links(DIMS), DIMS, mu, MW).toarray()
        ev = _sorted(np.linalg.eigvals(h))
        want = _sorted(np.repeat(z, 6))
        assert ev.shape == want.shape == (384,)
        assert np.abs(ev - want).max() < 1e-10, mu


def test_closed_form_reproduces_stored():
    for mu, z in _stored().items():
        now = freefield.spectrum(DIMS, mu, MW)
        assert np.abs(_sorted(now) - _sorted(z)).max() < 1e-14
