"""Wilson-Dirac operator and an unpreconditioned BiCGStab (oracle; test infrastructure).

Sec. 2 of the paper: N_f = 2 Wilson fermions at hopping parameter kappa; the
quark propagator S_F = M^{-1} of the Wilson matrix is obtained by Krylov solves
(Sec. 2: "mixed precision implementations of CG and BiCGstab").  The paper
states no sign conventions; the reading used throughout is the standard Wilson
matrix with Wilson parameter r = 1,

    M = 1 - kappa * D,
    (D psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                        + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ],

periodic in space and antiperiodic in time: a hop across the time boundary
(t = T-1 <-> t = 0) picks up the factor ``t_bc`` (-1).

The solver is textbook BiCGStab (van der Vorst 1992) on the full lattice,
with no even-odd preconditioning, so it shares nothing with the GPU path's
Schur-complement solve.
"""

from __future__ import annotations

import numpy as np

from .lattice import gammas, gamma5, site_axis, spinor_shape, volume


def _shift_forward(psi: np.ndarray, mu: int, t_bc: float) -> np.ndarray:
    """psi(x + mu) at every x, with the time boundary factor."""
    ax = site_axis(mu)
    out = np.roll(psi, -1, axis=ax)
    if mu == 3 and t_bc != 1:
        idx = [slice(None)] * out.ndim
        idx[ax] = -1  # sites with t = T-1 fetched psi(t = 0)
        out[tuple(idx)] *= t_bc
    return out


def _shift_backward(psi: np.ndarray, mu: int, t_bc: float) -> np.ndarray:
    """psi(x - mu) at every x, with the time boundary factor."""
    ax = site_axis(mu)
    out = np.roll(psi, 1, axis=ax)
    if mu == 3 and t_bc != 1:
        idx = [slice(None)] * out.ndim
        idx[ax] = 0  # sites with t = 0 fetched psi(t = T-1)
        out[tuple(idx)] *= t_bc
    return out


def _colour(u: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(U psi)[s, a] = sum_b U[a, b] psi[s, b] at every site."""
    return psi @ np.swapaxes(u, -1, -2)


def _spin(p: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """(P psi)[s, a] = sum_r P[s, r] psi[r, a] at every site."""
    return np.einsum("sr,...ra->...sa", p, psi)


def hop(U: np.ndarray, psi: np.ndarray, t_bc: float = -1.0) -> np.ndarray:
    """The Wilson hopping term D psi (full lattice, any leading batch axes on psi)."""
    g = gammas()
    one = np.eye(4, dtype=np.complex128)
    out = np.zeros(np.broadcast_shapes(psi.shape), dtype=np.complex128)
    for mu in range(4):
        u = U[..., mu, :, :]
        # forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
        out += _spin(one - g[mu], _colour(u, _shift_forward(psi, mu, t_bc)))
        # backward: (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu)
        u_back = np.roll(u, 1, axis=site_axis(mu)).conj().swapaxes(-1, -2)
        out += _spin(one + g[mu], _colour(u_back, _shift_backward(psi, mu, t_bc)))
    return out


def apply_m(U, psi, kappa, t_bc=-1.0):
    """M psi = psi - kappa D psi."""
    return psi - kappa * hop(U, psi, t_bc)


def apply_mdag(U, psi, kappa, t_bc=-1.0):
    """M^dagger psi, written as gamma_5 M gamma_5 psi (gamma5-hermiticity of M)."""
    g5 = gamma5()
    return _spin(g5, apply_m(U, _spin(g5, psi), kappa, t_bc))


def apply_gamma5(psi):
    return _spin(gamma5(), psi)


def dense_matrix(U, kappa, t_bc=-1.0, dims=None) -> np.ndarray:
    """M as a dense (12V x 12V) matrix; column j = M applied to unit vector j.

    Only for tiny lattices (a 4^4 lattice is 3072 x 3072).
    """
    if dims is None:
        lt, lz, ly, lx = U.shape[:4]
        dims = (lx, ly, lz, lt)
    n = 12 * volume(dims)
    unit = np.eye(n, dtype=np.complex128).reshape((n,) + spinor_shape(dims))
    cols = apply_m(U, unit, kappa, t_bc).reshape(n, n)
    return cols.T.copy()


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def bicgstab(apply_op, b, tol=1e-12, max_iter=10000, x0=None, max_restarts=20):
    """Solve A x = b by BiCGStab (van der Vorst 1992).

    Stops when the recursively updated residual satisfies ||r|| <= tol ||b||,
    then recomputes the true residual b - A x and restarts from the current
    iterate while that is still above tol.  Returns (x, info) where info has
    ``iters``, ``true_residual`` (relative) and ``converged``.
    """
    bnorm = np.sqrt(_dot(b, b).real)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if bnorm == 0.0:
        return x, dict(iters=0, true_residual=0.0, converged=True)
    total = 0
    for _ in range(max_restarts + 1):
        r = b - apply_op(x)
        if np.sqrt(_dot(r, r).real) <= tol * bnorm:
            break
        rhat = r.copy()
        rho = alpha = omega = 1.0 + 0j
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        while total < max_iter:
            rho_new = _dot(rhat, r)
            if rho_new == 0:
                break
            beta = (rho_new / rho) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = apply_op(p)
            alpha = rho_new / _dot(rhat, v)
            s = r - alpha * v
            t = apply_op(s)
            tt = _dot(t, t).real
            omega = _dot(t, s) / tt if tt > 0 else 0.0
            x = x + alpha * p + omega * s
            r = s - omega * t
            rho = rho_new
            total += 1
            if np.sqrt(_dot(r, r).real) <= tol * bnorm or omega == 0:
                break
        if total >= max_iter:
            break
    r = b - apply_op(x)
    res = float(np.sqrt(_dot(r, r).real) / bnorm)
    return x, dict(iters=total, true_residual=res, converged=bool(res <= tol))


def solve(U, b, kappa, t_bc=-1.0, tol=1e-12, max_iter=10000):
    """phi = M^{-1} b by full-lattice BiCGStab."""
    return bicgstab(lambda v: apply_m(U, v, kappa, t_bc), b, tol=tol, max_iter=max_iter)


def solve_adjoint(U, b, kappa, t_bc=-1.0, tol=1e-12, max_iter=10000):
    """chi = M^{-dagger} b by full-lattice BiCGStab on M^dagger."""
    return bicgstab(lambda v: apply_mdag(U, v, kappa, t_bc), b, tol=tol, max_iter=max_iter)


def plaquette(U) -> float:
    """Mean plaquette (1/3) Re Tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag."""
    acc = 0.0
    n = 0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            umu = U[..., mu, :, :]
            unu = U[..., nu, :, :]
            unu_xmu = np.roll(unu, -1, axis=site_axis(mu))
            umu_xnu = np.roll(umu, -1, axis=site_axis(nu))
            p = umu @ unu_xmu @ umu_xnu.conj().swapaxes(-1, -2) @ unu.conj().swapaxes(-1, -2)
            acc += np.trace(p, axis1=-2, axis2=-1).real.mean() / 3.0
            n += 1
    return float(acc / n)
