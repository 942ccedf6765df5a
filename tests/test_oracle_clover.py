"""Pins of the oracle's clover term (CPU)."""

import numpy as np

import synthetic
from oracle import clover, lattice, loops, wilson


def abelian_field(dims, n):
    """U_x = 1, U_y(x) = exp(i B x) 1 with B = 2 pi n / Lx, other links 1: every xy plaquette is exp(i B)."""
    lx, ly, lz, lt = dims
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (lt, lz, ly, lx, 4, 3, 3)).copy()
    B = 2 * np.pi * n / lx
    for x in range(lx):
        U[:, :, :, x, 1] = np.exp(1j * B * x) * np.eye(3)
    return U, B


def test_uniform_abelian_field_strength_is_sin_b():
    dims = (6, 4, 2, 4)
    U, B = abelian_field(dims, 1)
    F = clover.field_strength(U)
    assert np.abs(F[(0, 1)] - np.sin(B) * np.eye(3)).max() < 1e-14
    for plane, f in F.items():
        if plane != (0, 1):
            assert np.abs(f).max() < 1e-14
    # the clover term of that field: A = 1 - kappa c_sw sin(B) sigma_xy (x) 1.  With g_mu = [[0, X_mu],
    # [X_mu^dag, 0]], X_1 = i s_x, X_2 = -i s_y: g_1 g_2 = (-i s_z) (+) (-i s_z), so
    # sigma_12 = i g_1 g_2 = s_z (+) s_z = diag(1, -1, 1, -1)
    kappa, c_sw = 0.12, 1.3
    A = clover.clover_matrix(U, kappa, c_sw)
    sxy = clover.sigma(0, 1)
    assert np.allclose(sxy, np.diag([1, -1, 1, -1]), atol=1e-15)
    assert np.abs(A - (np.eye(12) - kappa * c_sw * np.sin(B) * np.kron(sxy, np.eye(3)))).max() < 1e-14


def test_clover_term_is_hermitian_commutes_with_gamma5_and_is_block_diagonal():
    dims = (4, 2, 2, 4)
    U = synthetic.gauge_field(dims, eps=0.45, seed=3)
    A = clover.clover_matrix(U, 0.12, 1.0)
    assert np.abs(A - np.conj(np.swapaxes(A, -1, -2))).max() < 1e-14
    g5 = np.kron(lattice.gamma5(), np.eye(3))
    assert np.abs(g5 @ A - A @ g5).max() < 1e-14
    assert np.abs(A[..., :6, 6:]).max() < 1e-15 and np.abs(A[..., 6:, :6]).max() < 1e-15
    # the field strength is traceless-antisymmetric in colour only through Q - Q^dag: hermitian
    for f in clover.field_strength(U).values():
        assert np.abs(f - np.conj(np.swapaxes(f, -1, -2))).max() < 1e-14


def test_free_field_and_c_sw_zero_give_the_wilson_matrix():
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, eps=0.45, seed=4)
    Ufree = np.broadcast_to(np.eye(3, dtype=np.complex128), U.shape).copy()
    assert np.abs(clover.clover_matrix(Ufree, 0.12, 1.7) - np.eye(12)).max() < 1e-14
    assert np.abs(clover.dense_matrix(U, 0.12, 0.0) - wilson.dense_matrix(U, 0.12)).max() == 0.0


def test_gauge_covariance_and_gamma5_hermiticity():
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, eps=0.45, seed=5)
    kappa, c_sw = 0.11, 1.2
    g = synthetic.random_gauge_transform(dims, seed=6)
    Ug = np.einsum("tzyxab,tzyxmbc->tzyxmac", g, U)
    for mu in range(4):
        Ug[..., mu, :, :] = Ug[..., mu, :, :] @ np.conj(np.swapaxes(np.roll(g, -1, axis=3 - mu), -1, -2))
    A, Ag = clover.clover_matrix(U, kappa, c_sw), clover.clover_matrix(Ug, kappa, c_sw)
    G = np.einsum("sr,tzyxab->tzyxsarb", np.eye(4), g).reshape(g.shape[:4] + (12, 12))
    assert np.abs(Ag - G @ A @ np.conj(np.swapaxes(G, -1, -2))).max() < 1e-13
    M = clover.dense_matrix(U, kappa, c_sw)
    g5 = np.kron(np.eye(32), np.kron(lattice.gamma5(), np.eye(3)))
    assert np.abs(g5 @ M @ g5 - np.conj(M.T)).max() < 1e-14
    # exact clover loops are gauge invariant
    Lc = np.linalg.inv(M)
    Lg = np.linalg.inv(clover.dense_matrix(Ug, kappa, c_sw))
    tr = lambda minv: np.array([np.trace(minv[12 * i:12 * i + 12, 12 * i:12 * i + 12]) for i in range(32)])
    assert np.abs(tr(Lc) - tr(Lg)).max() < 1e-12


def test_solver_matches_dense_inverse():
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, eps=0.45, seed=7)
    kappa, c_sw = 0.11, 1.5
    b = synthetic.random_spinor(dims, seed=8)
    x, info = clover.solve(U, b, kappa, c_sw, tol=1e-13)
    ref = np.linalg.solve(clover.dense_matrix(U, kappa, c_sw), b.ravel()).reshape(b.shape)
    assert info["converged"] and np.abs(x - ref).max() < 1e-11 * np.abs(ref).max()
