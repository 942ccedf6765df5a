"""Pins for the oracle's geometry and gamma algebra (CPU)."""

import numpy as np

from oracle import lattice


def test_clifford_algebra():
    g = lattice.gammas()
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)  # hermitian
        for n in range(4):
            anti = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(anti, 2 * np.eye(4) * (m == n))


def test_gamma5_chiral_and_g1g3_spin_off_diagonal():
    g5 = lattice.gamma5()
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    g = lattice.gammas()
    g13 = g[0] @ g[2]
    # Sec. 3: gamma_1 gamma_3 is strongly spin-off-diagonal "in this basis".
    assert np.allclose(np.diag(g13), 0)


def test_gamma_basis_is_orthogonal():
    b = lattice.gamma_basis()
    assert b.shape == (16, 4, 4)
    gram = np.einsum("iab,jab->ij", b.conj(), b)  # Tr[G_i^dag G_j]
    assert np.allclose(gram, 4 * np.eye(16))
    assert lattice.GAMMA_NAMES[5] == "g5" and np.allclose(b[5], lattice.gamma5())


def test_lexicographic_matches_flattening():
    dims = (4, 2, 6, 2)
    x, y, z, t = lattice.coordinates(dims)
    idx = lattice.lexicographic_index(x, y, z, t, dims)
    assert np.array_equal(idx.ravel(), np.arange(lattice.volume(dims)))
    par = lattice.parity(x, y, z, t)
    assert par.sum() * 2 == lattice.volume(dims)
