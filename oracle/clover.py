"""Clover (Sheikholeslami-Wohlert) term of the Wilson matrix (oracle; test infrastructure).

The paper's inversions use plain Wilson fermions (Sec. 2).  The clover term is
the lowest-ranked extension of the build's scope and is not part of the
paper's method, so the convention is stated here rather than read from it:

    M = A - kappa D,        A(x) = 1 - kappa c_sw sum_{mu < nu} sigma_{mu nu} F_{mu nu}(x),
    sigma_{mu nu} = (i / 2) [gamma_mu, gamma_nu]                  (hermitian),
    F_{mu nu}(x)  = (Q_{mu nu}(x) - Q_{mu nu}(x)^dag) / (8 i)      (hermitian),

with Q_{mu nu}(x) the sum of the four plaquette "leaves" of the mu-nu plane that
start and end at x, all traversed the same way (mu first, then nu).  A is
hermitian and commutes with gamma_5 (so M keeps gamma_5-hermiticity), and it
acts on one site only.  In the chiral basis every sigma_{mu nu} is
block-diagonal in the spin pairs (0, 1) and (2, 3), so A splits into two 6 x 6
blocks per site.  c_sw = 0 gives the Wilson matrix of ``wilson``.
"""

from __future__ import annotations

import numpy as np

from . import wilson
from .lattice import gammas


def _dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


def _at(f: np.ndarray, m: int, k: int) -> np.ndarray:
    """f(x + k m) at every x for a colour-matrix field [T][Z][Y][X][3][3] (periodic)."""
    return np.roll(f, -k, axis=3 - m)


def leaves(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """Q_{mu nu}(x): the four plaquettes around x in the mu-nu plane, [T][Z][Y][X][3][3]."""
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    # x -> x+mu -> x+mu+nu -> x+nu -> x
    q = Um @ _at(Un, mu, 1) @ _dag(_at(Um, nu, 1)) @ _dag(Un)
    # x -> x+nu -> x+nu-mu -> x-mu -> x
    q = q + Un @ _dag(_at(_at(Um, nu, 1), mu, -1)) @ _dag(_at(Un, mu, -1)) @ _at(Um, mu, -1)
    # x -> x-mu -> x-mu-nu -> x-nu -> x
    q = q + _dag(_at(Um, mu, -1)) @ _dag(_at(_at(Un, mu, -1), nu, -1)) @ _at(_at(Um, mu, -1), nu, -1) @ _at(Un, nu, -1)
    # x -> x-nu -> x-nu+mu -> x+mu -> x
    q = q + _dag(_at(Un, nu, -1)) @ _at(Um, nu, -1) @ _at(_at(Un, nu, -1), mu, 1) @ _dag(Um)
    return q


def field_strength(U: np.ndarray) -> dict:
    """F_{mu nu}(x) = (Q - Q^dag) / (8 i) for the six planes mu < nu: {(mu, nu): [T][Z][Y][X][3][3]}."""
    out = {}
    for mu in range(4):
        for nu in range(mu + 1, 4):
            q = leaves(U, mu, nu)
            out[(mu, nu)] = (q - _dag(q)) / 8j
    return out


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (i / 2) [gamma_mu, gamma_nu]."""
    g = gammas()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def clover_matrix(U: np.ndarray, kappa: float, c_sw: float) -> np.ndarray:
    """A(x) = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x): [T][Z][Y][X][12][12], index 3 spin + colour."""
    F = field_strength(U)
    shape = U.shape[:4]
    A = np.broadcast_to(np.eye(12, dtype=np.complex128), shape + (12, 12)).copy()
    for (mu, nu), f in F.items():
        s = sigma(mu, nu)
        A -= kappa * c_sw * np.einsum("ab,...ij->...aibj", s, f).reshape(shape + (12, 12))
    return A


def apply_clover(U, psi, kappa, c_sw):
    """A psi (site by site)."""
    A = clover_matrix(U, kappa, c_sw)
    flat = psi.reshape(psi.shape[:-2] + (12,))
    return np.einsum("...ij,...j->...i", A, flat).reshape(psi.shape)


def apply_m(U, psi, kappa, c_sw, t_bc=-1.0):
    """M psi = A psi - kappa D psi."""
    return apply_clover(U, psi, kappa, c_sw) - kappa * wilson.hop(U, psi, t_bc)


def dense_matrix(U, kappa, c_sw, t_bc=-1.0) -> np.ndarray:
    """M as a dense 12V x 12V matrix (tiny lattices only)."""
    lt, lz, ly, lx = U.shape[:4]
    n = 12 * lx * ly * lz * lt
    unit = np.eye(n, dtype=np.complex128).reshape((n, lt, lz, ly, lx, 4, 3))
    return apply_m(U, unit, kappa, c_sw, t_bc).reshape(n, n).T.copy()


def solve(U, b, kappa, c_sw, t_bc=-1.0, tol=1e-12, max_iter=10000):
    """phi = M^{-1} b by full-lattice BiCGStab."""
    A = clover_matrix(U, kappa, c_sw)

    def op(v):
        flat = v.reshape(v.shape[:-2] + (12,))
        return np.einsum("...ij,...j->...i", A, flat).reshape(v.shape) - kappa * wilson.hop(U, v, t_bc)

    return wilson.bicgstab(op, b, tol=tol, max_iter=max_iter)
