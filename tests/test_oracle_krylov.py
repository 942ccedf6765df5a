"""Pins of the oracle's Schur system and fixed-iteration Krylov maps (CPU).

Each check uses something outside the oracle's own formulas: the dense matrix's
parity blocks, numpy's least-squares and linear solvers, or a closed form.
"""

import numpy as np
import pytest

import synthetic
from oracle import krylov, lattice, wilson


def _parity_of_index(dims):
    x, y, z, t = lattice.coordinates(dims)
    par = lattice.parity(x, y, z, t)  # [T][Z][Y][X]
    return np.repeat(par.ravel(), 12)  # the dense matrix's index order: site, spin, colour


@pytest.mark.parametrize("kappa", [0.11, 0.16])
def test_schur_operator_is_the_dense_schur_complement(kappa):
    dims = (2, 2, 2, 4)
    U = synthetic.gauge_field(dims, eps=0.5, seed=3)
    M = wilson.dense_matrix(U, kappa, -1.0)
    par = _parity_of_index(dims)
    e, o = np.where(par == 0)[0], np.where(par == 1)[0]
    assert np.allclose(M[np.ix_(o, o)], np.eye(len(o)), atol=0, rtol=0)  # D only links opposite parities
    S = M[np.ix_(e, e)] - M[np.ix_(e, o)] @ M[np.ix_(o, e)]
    n = 12 * lattice.volume(dims)
    unit = np.eye(n, dtype=np.complex128)[e].reshape((len(e),) + lattice.spinor_shape(dims))
    cols = krylov.schur_apply(U, unit, kappa).reshape(len(e), n)[:, e]
    assert np.abs(cols.T - S).max() < 1e-14
    cols_dag = krylov.schur_apply_dag(U, unit, kappa).reshape(len(e), n)[:, e]
    assert np.abs(cols_dag.T - S.conj().T).max() < 1e-14


def test_schur_rhs_and_reconstruction_give_the_solution():
    dims, kappa = (2, 2, 2, 4), 0.13
    U = synthetic.gauge_field(dims, eps=0.5, seed=5)
    b = synthetic.random_spinor(dims, seed=7, n=1)[0]
    x = np.linalg.solve(wilson.dense_matrix(U, kappa), b.ravel()).reshape(b.shape)
    ev = krylov.parity_mask(dims, 0)
    xe = krylov.project(x, ev)
    bhat = krylov.schur_rhs(U, b, kappa)
    assert np.abs(krylov.schur_apply(U, xe, kappa) - bhat).max() < 1e-13
    assert np.abs(krylov.schur_reconstruct(U, xe, b, kappa) - x).max() < 1e-13


def _small_system(n=12, seed=0):
    rng = np.random.default_rng(seed)
    A = np.eye(n) + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return A, b


def test_cgnr_iterates_are_krylov_least_squares_minimisers():
    """CGNR's k-th iterate minimises |b - A x| over K_k(A^dag A, A^dag b)."""
    A, b = _small_system()
    Ah = A.conj().T
    for k in range(1, 7):
        xk, info = krylov.cgnr(lambda v: A @ v, lambda v: Ah @ v, b, n_iter=k)
        assert info["iters"] == k
        basis = [Ah @ b]
        for _ in range(k - 1):
            basis.append(Ah @ (A @ basis[-1]))
        K = np.stack(basis, axis=1)
        c, *_ = np.linalg.lstsq(A @ K, b, rcond=None)
        ref = K @ c
        assert np.linalg.norm(xk - ref) < 1e-10 * np.linalg.norm(ref)


def test_cgnr_converges_to_the_solution():
    A, b = _small_system(seed=1)
    x, info = krylov.cgnr(lambda v: A @ v, lambda v: A.conj().T @ v, b, tol=1e-13)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) < 1e-11 * np.linalg.norm(ref)
    assert info["residual"] <= 1e-13


def test_bicgstab_fixed_first_iterate_closed_form():
    """x_1 = alpha b + omega s, alpha = <b,b>/<b,Ab>, s = b - alpha A b, omega = <As,s>/<As,As>."""
    A, b = _small_system(seed=2)
    x1, r1 = krylov.bicgstab_fixed(lambda v: A @ v, b, 1)
    alpha = np.vdot(b, b) / np.vdot(b, A @ b)
    s = b - alpha * (A @ b)
    t = A @ s
    omega = np.vdot(t, s) / np.vdot(t, t)
    assert np.linalg.norm(x1 - (alpha * b + omega * s)) < 1e-14 * np.linalg.norm(x1)
    assert np.linalg.norm(r1 - (b - A @ x1)) < 1e-13 * np.linalg.norm(b)


def test_bicgstab_fixed_residual_recursion_and_convergence():
    A, b = _small_system(seed=3)
    for k in (2, 5, 9):
        xk, rk = krylov.bicgstab_fixed(lambda v: A @ v, b, k)
        assert np.linalg.norm(rk - (b - A @ xk)) < 1e-12 * np.linalg.norm(b)
    x, r = krylov.bicgstab_fixed(lambda v: A @ v, b, 40)
    assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)


def test_krylov_maps_on_the_schur_system():
    """On a lattice Schur system both maps approach M^-1 b after reconstruction."""
    dims, kappa = (2, 2, 2, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=8)
    b = synthetic.random_spinor(dims, seed=9, n=1)[0]
    ref = np.linalg.solve(wilson.dense_matrix(U, kappa), b.ravel()).reshape(b.shape)
    bhat = krylov.schur_rhs(U, b, kappa)
    op = lambda v: krylov.schur_apply(U, v, kappa)  # noqa: E731
    opd = lambda v: krylov.schur_apply_dag(U, v, kappa)  # noqa: E731
    xe, _ = krylov.cgnr(op, opd, bhat, tol=1e-13)
    assert np.abs(krylov.schur_reconstruct(U, xe, b, kappa) - ref).max() < 1e-11 * np.abs(ref).max()
    xe, _ = krylov.bicgstab_fixed(op, bhat, 60)
    assert np.abs(krylov.schur_reconstruct(U, xe, b, kappa) - ref).max() < 1e-11 * np.abs(ref).max()
