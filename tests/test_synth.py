"""Input generators: Philox known answers and the SU(3) property of links."""

import numpy as np

import synth


def test_philox_known_answers():
    """Known-answer vectors published with Philox4x32-10 (Random123)."""
    f = synth.philox4x32_10
    assert [int(v) for v in f(0, 0, 0, 0, 0, 0)] == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    m = 0xFFFFFFFF
    assert [int(v) for v in f(m, m, m, m, m, m)] == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    out = f(0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344, 0xA4093822, 0x299F31D0)
    assert [int(v) for v in out] == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_uniform_open_interval():
    u = synth.philox_uniform52(np.array([0, 0xFFFFFFFF]), np.array([0, 0xFFFFFFFF]))
    assert np.all(u > 0) and np.all(u < 1)


def test_links_are_su3_and_seeded():
    dims = (4, 2, 2, 2)
    u = synth.gauge_links(dims, 7, 0.6).reshape(-1, 3, 3)
    eye = np.einsum("lab,lcb->lac", u, u.conj())
    assert np.abs(eye - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(u) - 1).max() < 1e-14
    assert np.array_equal(u, synth.gauge_links(dims, 7, 0.6).reshape(-1, 3, 3))
    assert not np.allclose(u, synth.gauge_links(dims, 8, 0.6).reshape(-1, 3, 3))
    # eps sets the distance from the identity
    d1 = np.abs(synth.gauge_links(dims, 7, 0.1).reshape(-1, 3, 3) - np.eye(3)).mean()
    assert d1 < np.abs(u - np.eye(3)).mean()


def test_vectors_unit_norm():
    x = synth.gaussian_vectors(120, 3, 2)
    assert np.allclose(np.linalg.norm(x, axis=1), 1)
    w = synth.plane_wave_vectors((2, 2, 2, 4), [(1, 0, 0, 1)], 3)
    assert w.shape == (1, 12 * 32) and np.isclose(np.linalg.norm(w), 1)


def test_batched_instance_recipe():
    """Sizes cycle 4^4/6^4/8^4, mu cycles 0.1/0.2/0.3, eps in [0.5, 0.7],
    right-hand-side counts in 1..16 and uneven, all reproducible."""
    a = synth.batched_instances(32)
    assert a == synth.batched_instances(32)
    for i, d in enumerate(a):
        assert d["dims"] == [(4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 8)][i % 3]
        assert d["mu"] == (0.1, 0.2, 0.3)[i % 3]
        assert 0.5 <= d["eps"] <= 0.7 and 1 <= d["nrhs"] <= 16
        assert d["gauge_seed"] == 100 + i and d["source_seed"] == 200 + i
    assert len({d["nrhs"] for d in a}) > 5
    r, l, lam = synth.synthetic_deflation(96, 7, 3)
    assert r.shape == (96, 7) and l.shape == (96, 7) and lam.shape == (7,)
    assert np.all(np.abs(lam.real) >= 0.05) and np.all(np.abs(lam.real) <= 0.5)
