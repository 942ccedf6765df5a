"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module only *draws* inputs: gauge links, random spinor fields and random
gauge transformations.  It holds none of the disconnected-loop method's
arithmetic (no Dirac operator, no solver, no noise map, no contraction), so the
CUDA path and the oracle can both take their inputs from here without sharing
any of the computation they are compared on.

Array conventions (the canonical host layout of the C ABI):

* a lattice has extents ``dims = (Lx, Ly, Lz, T)``; arrays are indexed
  ``[t, z, y, x, ...]`` so that flattening gives the lexicographic site index
  ``i = x + Lx*(y + Ly*(z + Lz*t))`` with x fastest;
* a gauge field is ``complex128[T, Lz, Ly, Lx, 4, 3, 3]`` holding ``U_mu(x)``
  with ``mu = 0..3`` for the x, y, z, t directions and ``U[a, b]`` row ``a``,
  column ``b``;
* a spinor field is ``complex128[..., T, Lz, Ly, Lx, 4, 3]`` (spin, then colour).

The ensemble of the paper (Sec. 2: N_f=2 Wilson, beta=5.6, 16^3x32, SESAM) is not
available, so links are drawn near the identity, ``U = exp(i*eps*H)`` with
``H = sum_a h_a lambda_a / 2`` and ``h_a ~ N(0, 1)``; ``eps`` sets the mean
plaquette (eps = 0.45 gives about 0.57, eps = 0.30 about 0.79).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "gauge_field",
    "unit_gauge",
    "random_su3",
    "random_spinor",
    "random_gauge_transform",
    "lattice_volume",
    "WORKLOADS",
]


def lattice_volume(dims) -> int:
    lx, ly, lz, lt = dims
    return int(lx) * int(ly) * int(lz) * int(lt)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices lambda_1..lambda_8 as complex128[8, 3, 3]."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _rng(seed: int, stream: int) -> np.random.Generator:
    # A counter-based bit generator keyed by (seed, stream): independent draws for
    # links, spinors and transformations with the same seed.
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


def _exp_i_hermitian(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*H) for a batch of Hermitian 3x3 matrices, by eigendecomposition."""
    w, v = np.linalg.eigh(h)
    phase = np.exp(1j * eps * w)
    return np.einsum("...ij,...j,...kj->...ik", v, phase, v.conj())


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Project onto SU(3): Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1)."""
    r0 = u[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = u[..., 1, :]
    r1 = r1 - np.sum(r0.conj() * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.cross(r0, r1).conj()
    return np.stack([r0, r1, r2], axis=-2)


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Near-identity SU(3) links U_mu(x) = exp(i*eps*H), H = sum_a h_a lambda_a/2."""
    lx, ly, lz, lt = (int(d) for d in dims)
    g = _rng(seed, 1)
    h = g.standard_normal(size=(lt, lz, ly, lx, 4, 8))
    herm = np.einsum("...a,aij->...ij", h, gell_mann()) / 2.0
    return _reunitarise(_exp_i_hermitian(herm, eps))


def unit_gauge(dims) -> np.ndarray:
    """The free field U_mu(x) = 1."""
    lx, ly, lz, lt = (int(d) for d in dims)
    u = np.zeros((lt, lz, ly, lx, 4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def random_su3(shape, seed: int, stream: int = 3) -> np.ndarray:
    """Broadly distributed SU(3) matrices (exp of a unit-scale Hermitian matrix)."""
    g = _rng(seed, stream)
    h = g.standard_normal(size=tuple(shape) + (8,))
    herm = np.einsum("...a,aij->...ij", h, gell_mann()) * 1.5
    return _reunitarise(_exp_i_hermitian(herm, 1.0))


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """A site-dependent SU(3) matrix g(x), complex128[T, Lz, Ly, Lx, 3, 3]."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return random_su3((lt, lz, ly, lx), seed, stream=3)


def random_spinor(dims, seed: int, n: int | None = None) -> np.ndarray:
    """Gaussian complex spinor field(s), complex128[(n,) T, Lz, Ly, Lx, 4, 3]."""
    lx, ly, lz, lt = (int(d) for d in dims)
    shape = (lt, lz, ly, lx, 4, 3) if n is None else (int(n), lt, lz, ly, lx, 4, 3)
    g = _rng(seed, 2)
    return (g.standard_normal(size=shape) + 1j * g.standard_normal(size=shape)) / np.sqrt(2.0)


# The workloads: the shapes and parameters of the paper's lattice (Sec. 2) with
# synthetic links.  kappa = 0.157 on uncorrelated eps = 0.45 links is past the
# critical hopping parameter (the Wilson matrix has eigenvalues with negative
# real part and BiCGStab does not converge), so the eps = 0.45 workloads run at
# kappa = 0.140 and the kappa = 0.157 variant uses rougher links, eps = 0.60.
WORKLOADS = {
    # 4^4 exact loops, all 12V point sources
    "exact_4x4x4x4": dict(dims=(4, 4, 4, 4), kappa=0.10, eps=0.30, seed=1, tol=1e-12),
    # the paper's lattice shape, near-identity links with plaquette ~0.57
    "wilson_16x16x16x32": dict(dims=(16, 16, 16, 32), kappa=0.140, eps=0.45, seed=1, tol=1e-10),
    "wilson_16x16x16x32_k157": dict(dims=(16, 16, 16, 32), kappa=0.157, eps=0.60, seed=1, tol=1e-10),
    # truncated-solver study lattice
    "tsm_8x8x8x16": dict(dims=(8, 8, 8, 16), kappa=0.140, eps=0.45, seed=1, tol=1e-10),
    "tsm_8x8x8x16_k157": dict(dims=(8, 8, 8, 16), kappa=0.157, eps=0.60, seed=1, tol=1e-10),
    # supercritical: kept to test that the solver stops cleanly
    "supercritical_8x8x8x16": dict(dims=(8, 8, 8, 16), kappa=0.157, eps=0.45, seed=1, tol=1e-10),
}
