"""Even-site Schur system and fixed-iteration Krylov maps (oracle; test infrastructure).

The truncated solver method (Sec. 2) needs a deterministic low-precision map
f_LP(eta), which approximates M^{-1} eta.  The map is the result of a Krylov
solver run for a given number of iterations (or to a loose tolerance), so it
depends on the solver's steps, not only on M.  This module restates those
steps so that the GPU solver can be compared with them iteration for
iteration:

* the even-odd Schur complement of M = 1 - kappa D, written with parity
  projectors on full-lattice fields (no even-odd storage):
      Mhat   = P_e (1 - kappa^2 D P_o D) P_e,
      bhat   = P_e (b + kappa D P_o b),
      x_o    = P_o (b + kappa D x_e);
* CG on the normal equations (CGNR), the single-precision solver Sec. 2 names
  for the low-precision inversions.  It follows Hestenes & Stiefel's CG
  applied to A^dag A x = A^dag b, tracking the residual r = b - A x of the
  original system (Saad, Iterative Methods for Sparse Linear Systems,
  Algorithm 8.4);
* BiCGStab (van der Vorst 1992) for a fixed number of iterations from x = 0
  with shadow residual rhat = b.

Pins (tests/test_oracle_krylov.py):

* The Schur operator equals M_ee - M_eo M_oe, built from the dense matrix's
  parity blocks (M_oo = 1).
* CGNR's k-th iterate equals the least-squares minimiser of |b - A x| over the
  Krylov space K_k(A^dag A, A^dag b), computed by numpy's lstsq.
* BiCGStab's first iterate has a closed form.  Its recursive residual equals
  the true residual b - A x_k, and it converges to numpy's solve on small
  systems.
"""

from __future__ import annotations

import numpy as np

from .lattice import coordinates, parity
from .wilson import hop


def parity_mask(dims, p: int) -> np.ndarray:
    """Boolean [T][Z][Y][X] mask of the sites with (x+y+z+t) & 1 == p."""
    x, y, z, t = coordinates(dims)
    return parity(x, y, z, t) == p


def project(psi: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """psi on the sites of `mask`, zero elsewhere (fields [..., T, Z, Y, X, 4, 3])."""
    return psi * mask[..., None, None]


def schur_apply(U, xe, kappa, t_bc=-1.0):
    """Mhat x_e = x_e - kappa^2 P_e D P_o D x_e (x_e supported on even sites)."""
    dims = xe.shape[-6:-2][::-1]
    ev, od = parity_mask(dims, 0), parity_mask(dims, 1)
    xe = project(xe, ev)
    return xe - kappa * kappa * project(hop(U, project(hop(U, xe, t_bc), od), t_bc), ev)


def schur_apply_dag(U, xe, kappa, t_bc=-1.0):
    """Mhat^dag x_e = x_e - kappa^2 P_e D^dag P_o D^dag x_e, with D^dag = g5 D g5."""
    g5 = np.array([1.0, 1.0, -1.0, -1.0])[:, None]
    dims = xe.shape[-6:-2][::-1]
    ev, od = parity_mask(dims, 0), parity_mask(dims, 1)
    ddag = lambda v: g5 * hop(U, g5 * v, t_bc)  # noqa: E731
    xe = project(xe, ev)
    return xe - kappa * kappa * project(ddag(project(ddag(xe), od)), ev)


def schur_rhs(U, b, kappa, t_bc=-1.0):
    """bhat = P_e (b + kappa D P_o b)."""
    dims = b.shape[-6:-2][::-1]
    ev, od = parity_mask(dims, 0), parity_mask(dims, 1)
    return project(b + kappa * hop(U, project(b, od), t_bc), ev)


def schur_reconstruct(U, xe, b, kappa, t_bc=-1.0):
    """Full solution from x_e: x = x_e + P_o (b + kappa D x_e)."""
    dims = b.shape[-6:-2][::-1]
    ev, od = parity_mask(dims, 0), parity_mask(dims, 1)
    xe = project(xe, ev)
    return xe + project(b + kappa * hop(U, xe, t_bc), od)


def _dot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def cgnr(apply_a, apply_adag, b, n_iter=None, tol=None, max_iter=100000):
    """CG on A^dag A x = A^dag b from x = 0, tracking r = b - A x.

    Runs exactly `n_iter` iterations, or (with `tol`) until |r| <= tol |b|.
    Returns (x, info) with ``iters`` and the recursive ``residual`` |r|/|b|.
    """
    x = np.zeros_like(b)
    r = b.copy()
    z = apply_adag(r)
    p = z.copy()
    zz = _dot(z, z).real
    bnorm = np.sqrt(_dot(b, b).real)
    k = 0
    limit = n_iter if n_iter is not None else max_iter
    while k < limit:
        if tol is not None and np.sqrt(_dot(r, r).real) <= tol * bnorm:
            break
        if zz == 0.0:
            break
        w = apply_a(p)
        alpha = zz / _dot(w, w).real
        x = x + alpha * p
        r = r - alpha * w
        z = apply_adag(r)
        zz_new = _dot(z, z).real
        p = z + (zz_new / zz) * p
        zz = zz_new
        k += 1
    return x, dict(iters=k, residual=float(np.sqrt(_dot(r, r).real) / bnorm) if bnorm > 0 else 0.0)


def bicgstab_fixed(apply_a, b, n_iter: int):
    """n_iter BiCGStab iterations from x = 0 with rhat = r_0 = b (no restarts).

    Returns (x, r) with r the recursively updated residual.  Stops early only
    if an iteration produces an exactly zero residual or t = 0.
    """
    x = np.zeros_like(b)
    r = b.copy()
    rhat = b.copy()
    p = r.copy()
    rho = _dot(rhat, r)
    for _ in range(n_iter):
        v = apply_a(p)
        alpha = rho / _dot(rhat, v)
        s = r - alpha * v
        t = apply_a(s)
        tt = _dot(t, t).real
        if tt == 0.0:
            x = x + alpha * p
            r = s
            break
        omega = _dot(t, s) / tt
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_new = _dot(rhat, r)
        if rho_new == 0:
            break
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        rho = rho_new
    return x, r
