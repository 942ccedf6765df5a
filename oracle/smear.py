"""Gauge-covariant Gaussian smearing (oracle; test infrastructure).

Sec. 2 of the paper: smeared quark fields are built with gauge-covariant
Gaussian smearing for a range of smearing parameters (values not given).
Reading: the Wuppertal/Gaussian form

    K = [ (1 + alpha * H) / (1 + 6 alpha) ]^n,
    (H psi)(x) = sum_{j = x, y, z} [ U_j(x) psi(x + j) + U_j(x - j)^dagger psi(x - j) ],

a purely spatial (3-d) operator, periodic in space, acting on colour only
(each spin component separately), with unsmoothed links.  The 1/(1 + 6 alpha)
normalisation makes K = 1 on a constant field in the free theory.
"""

from __future__ import annotations

import numpy as np

from .lattice import site_axis


def hop3(U: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """The spatial hopping operator H psi (no spin structure, periodic)."""
    out = np.zeros(psi.shape, dtype=np.complex128)
    for j in range(3):
        ax = site_axis(j)
        u = U[..., j, :, :]
        fwd = np.roll(psi, -1, axis=ax)
        out += fwd @ np.swapaxes(u, -1, -2)
        u_back = np.roll(u, 1, axis=ax).conj().swapaxes(-1, -2)
        bwd = np.roll(psi, 1, axis=ax)
        out += bwd @ np.swapaxes(u_back, -1, -2)
    return out


def smear(U: np.ndarray, psi: np.ndarray, alpha: float, n_iter: int) -> np.ndarray:
    """K psi with K = [(1 + alpha H)/(1 + 6 alpha)]^n_iter."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    for _ in range(n_iter):
        out = (out + alpha * hop3(U, out)) / (1.0 + 6.0 * alpha)
    return out
