"""Pins of the oracle's momentum loops and correlators (CPU)."""

import numpy as np

import synthetic
from oracle import correlators, lattice, loops, wilson

G16 = lattice.gamma_basis()


def test_zero_momentum_loops_are_the_loops():
    dims = (4, 2, 2, 4)
    eta = synthetic.random_spinor(dims, seed=1, n=3)
    phi = synthetic.random_spinor(dims, seed=2, n=3)
    got = correlators.momentum_loops(eta, phi, [(0, 0, 0), (1, 0, 1)], G16)
    assert np.abs(got[:, 0] - loops.stochastic_loops(eta, phi)).max() < 1e-12
    # a plane wave at p: the momentum sum equals the zero-momentum sum of the phase-weighted field
    ph = correlators.momentum_phases(dims, [(1, 0, 1)])[0]
    ref = loops.stochastic_loops(eta, phi * ph[None, ..., None, None])
    assert np.abs(got[:, 1] - ref).max() < 1e-12


def test_exact_momentum_loops_zero_momentum_and_translation():
    dims, kappa = (4, 2, 2, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.5, seed=3)
    moms = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (1, 1, 1)]
    L = correlators.exact_momentum_loops_dense(U, kappa, moms, G16)
    assert np.abs(L[0] - loops.exact_loops_dense(U, kappa, -1.0)).max() < 1e-12
    # U'(x) = U(x + e_x): M'^-1(x, x) = M^-1(x + e_x, x + e_x), so L'(p) = exp(+i p_x) L(p)
    Us = np.roll(U, -1, axis=3)  # U has shape [T][Z][Y][X][mu][3][3]
    Lt = correlators.exact_momentum_loops_dense(Us, kappa, moms, G16)
    for i, n in enumerate(moms):
        assert np.abs(Lt[i] - np.exp(2j * np.pi * n[0] / dims[0]) * L[i]).max() < 1e-11


def test_free_field_has_no_loops_at_nonzero_momentum():
    dims, kappa = (4, 2, 2, 4), 0.1
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, 2, 2, 4, 4, 3, 3)).copy()
    L = correlators.exact_momentum_loops_dense(U, kappa, [(0, 0, 0), (1, 0, 0), (2, 1, 1)], G16)
    assert np.abs(L[0, 0]).min() > 1.0
    assert np.abs(L[1:]).max() < 1e-12


def test_disconnected_equals_fft_cross_correlation():
    """Eq. 3 read as a product of traces is a circular cross-correlation in t:
    numpy's FFT gives it as ifft(fft(L_B) * conj(fft(conj(L_A)))), with no loop over t."""
    rng = np.random.default_rng(0)
    T = 7
    lb = rng.standard_normal((3, T)) + 1j * rng.standard_normal((3, T))
    la = rng.standard_normal((3, T)) + 1j * rng.standard_normal((3, T))
    D = correlators.disconnected(lb, la, spatial_volume=8)
    ref = -np.fft.ifft(np.fft.fft(lb, axis=-1) * np.conj(np.fft.fft(np.conj(la), axis=-1)), axis=-1) / (8 * T)
    assert np.abs(D - ref).max() < 1e-14 * np.abs(ref).max()
    # dt = 1 on T = 2 by hand: L_B(1) L_A(0) + L_B(0) L_A(1)
    d2 = correlators.disconnected(np.array([2.0, 3.0]), np.array([5.0, 7.0]), spatial_volume=1)
    assert np.allclose(d2, [-(2 * 5 + 3 * 7) / 2, -(3 * 5 + 2 * 7) / 2], rtol=1e-15)


def _connected_from_dense(minv, dims, src, momenta, gammas16):
    """Eq. 1 with the source sum replaced by the single point y = src, read straight off
    the dense inverse: S(x; y) = M^-1 block (x, y), S(y; x) = M^-1 block (y, x), no
    gamma5-hermiticity.  C^{BA}(p, t) = -sum_{x: x_4 = y_4 + t} exp(-i p.(x - y))
    Tr[S(y; x) Gamma_B S(x; y) Gamma_A].  Returns [P][16 A][16 B][T]."""
    lx, ly, lz, lt = dims
    V = lx * ly * lz * lt
    iy = int(lattice.lexicographic_index(src[0], src[1], src[2], src[3], dims))
    out = np.zeros((len(momenta), 16, 16, lt), dtype=np.complex128)
    g = [np.kron(gammas16[k], np.eye(3)) for k in range(16)]
    for ix in range(V):
        x = (ix % lx, (ix // lx) % ly, (ix // (lx * ly)) % lz, ix // (lx * ly * lz))
        s_xy = minv[12 * ix:12 * ix + 12, 12 * iy:12 * iy + 12]
        s_yx = minv[12 * iy:12 * iy + 12, 12 * ix:12 * ix + 12]
        t = (x[3] - src[3]) % lt
        for q, n in enumerate(momenta):
            arg = 2 * np.pi * sum(n[k] * (x[k] - src[k]) / dims[k] for k in range(3))
            ph = np.exp(-1j * arg)
            for A in range(16):
                left = s_xy @ g[A] @ s_yx  # S(x;y) G_A S(y;x); Tr[S(y;x) G_B S(x;y) G_A] = Tr[G_B left]
                for B in range(16):
                    out[q, A, B, t] -= ph * np.sum(g[B].T * left)
    return out


def test_connected_all_gamma_pairs_from_the_dense_inverse():
    """Every (Gamma_A, Gamma_B) pair of Eq. 1 at p = 0 and p != 0 on a gauge field: the oracle's
    gamma5-hermiticity evaluation from the 12 point-source columns equals the trace of the two
    dense-inverse blocks S(y; x), S(x; y) taken as printed.  A swap of Gamma_A and Gamma_B, or a
    dagger on either, changes the non-symmetric pairs and fails this."""
    dims, kappa, src = (4, 2, 2, 4), 0.12, (1, 0, 1, 2)
    U = synthetic.gauge_field(dims, eps=0.45, seed=31)
    minv = np.linalg.inv(wilson.dense_matrix(U, kappa, -1.0, dims))
    moms = [(0, 0, 0), (1, 0, 0), (1, 1, 1)]
    ref = _connected_from_dense(minv, dims, src, moms, G16)
    iy = int(lattice.lexicographic_index(src[0], src[1], src[2], src[3], dims))
    lx, ly, lz, lt = dims
    # prop[j = 3 alpha + a][t][z][y][x][beta][b] = M^-1[(x, beta, b), (y, alpha, a)]
    prop = minv[:, 12 * iy:12 * iy + 12].T.reshape(12, lt, lz, ly, lx, 4, 3)
    got = correlators.connected(prop, src, moms, G16)
    floor = 1e-6 * np.linalg.norm(ref[0, 5, 5])
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.maximum(np.linalg.norm(ref, axis=-1), floor)
    assert (num / den).max() < 1e-10
    # the pairs are not symmetric in (A, B): the test sees an exchange of the two operators
    asym = np.linalg.norm(ref - np.swapaxes(ref, 1, 2), axis=-1) / den
    assert (asym > 1e-3).sum() > 100
    # nor symmetric under Gamma_A -> Gamma_A^dag for the anti-hermitian members of the basis
    herm = [k for k in range(16) if np.allclose(G16[k], G16[k].conj().T)]
    assert len(herm) == 6 and set(herm) == {0, 1, 2, 3, 4, 5}


def test_free_point_propagator_fft_equals_the_solver():
    dims, kappa, src = (4, 4, 2, 4), 0.11, (1, 2, 0, 3)
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, 2, 4, 4, 4, 3, 3)).copy()
    solved = correlators.point_propagator(U, kappa, src)
    fft = correlators.free_point_propagator(dims, kappa, src)
    assert np.abs(solved - fft).max() < 1e-11 * np.abs(fft).max()


def test_connected_pion_is_minus_sum_of_squares_and_symmetric():
    dims, kappa, src = (4, 4, 2, 4), 0.11, (0, 0, 0, 0)
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, 2, 4, 4, 4, 3, 3)).copy()
    prop = correlators.free_point_propagator(dims, kappa, src)
    C = correlators.connected(prop, src, [(0, 0, 0), (1, 0, 0)], G16)
    pion = C[0, 5, 5]  # Gamma_A = Gamma_B = gamma5
    direct = -np.array([np.sum(np.abs(prop[:, t]) ** 2) for t in range(dims[3])])
    assert np.abs(pion - direct).max() < 1e-12 * np.abs(direct).max()
    assert np.abs(pion.imag).max() < 1e-14 * np.abs(direct).max()
    assert np.allclose(pion[1:], pion[1:][::-1], rtol=1e-10)  # C(t) = C(T - t) for a free field
    # gauge links: the same reduction holds configuration by configuration
    Ug = synthetic.gauge_field(dims, eps=0.4, seed=5)
    pg = correlators.point_propagator(Ug, kappa, (1, 0, 1, 2))
    Cg = correlators.connected(pg, (1, 0, 1, 2), [(0, 0, 0)], G16)
    direct = -np.array([np.sum(np.abs(pg[:, t]) ** 2) for t in range(dims[3])])
    assert np.abs(Cg[0, 5, 5] - np.roll(direct, -2)).max() < 1e-12 * np.abs(direct).max()
    assert wilson.plaquette(Ug) < 0.99


def test_disconnected_pairs_reduces_to_the_product_formula():
    """With identical per-noise loops and full coverage the pair average is the plain product."""
    rng = np.random.default_rng(4)
    Q, T = 3, 4
    L = rng.standard_normal((Q, 16, T)) + 1j * rng.standard_normal((Q, 16, T))
    minus = [0, 2, 1]
    D = correlators.disconnected_pairs(np.stack([L] * 3), None, minus, spatial_volume=8)
    for q in range(Q):
        for A in (0, 5, 9):
            for B in (0, 5, 14):
                ref = correlators.disconnected(L[q, B], L[minus[q], A], 8)
                assert np.allclose(D[q, A, B], ref, rtol=1e-13, atol=1e-15)


def test_disconnected_pairs_excludes_self_products():
    """Two noise vectors: only the cross products n != m enter, each ordered pair once."""
    T = 2
    L = np.zeros((2, 1, 16, T), dtype=np.complex128)
    L[0, 0, 0] = [1.0, 2.0]
    L[1, 0, 0] = [3.0, 5.0]
    D = correlators.disconnected_pairs(L, None, [0], spatial_volume=1)
    # dt = 0: t = 0 -> (1*3 + 3*1)/2, t = 1 -> (2*5 + 5*2)/2; dt = 1: t = 0 -> (L(1) L(0)): (2*3 + 5*1)/2, t = 1 -> (1*5 + 3*2)/2
    assert np.isclose(D[0, 0, 0, 0], -(3.0 + 10.0) / 2)
    assert np.isclose(D[0, 0, 0, 1], -((6.0 + 5.0) / 2 + (5.0 + 6.0) / 2) / 2)
