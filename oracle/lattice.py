"""Lattice geometry, gamma matrices and the Gamma basis (oracle; test infrastructure).

Geometry (Sec. 2: a 16^3 x 32 lattice; periodic in space, antiperiodic in time
for the quark fields).  ``dims = (Lx, Ly, Lz, T)``; fields are numpy arrays
indexed ``[..., t, z, y, x, spin, colour]``.  Direction ``mu = 0, 1, 2, 3`` is
x, y, z, t and lives on array axis ``-6 + (3 - mu)`` of a spinor field.

Gamma matrices.  The paper names no basis ("in this basis", Sec. 3, about the
spin-off-diagonal gamma_1 gamma_3).  The reading taken here is the chiral
DeGrand-Rossi basis, in which gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 =
diag(1, 1, -1, -1) and gamma_1 gamma_3 has no diagonal spin entries, which is
consistent with that remark.
"""

from __future__ import annotations

import numpy as np


def volume(dims) -> int:
    lx, ly, lz, lt = dims
    return int(lx * ly * lz * lt)


def spinor_shape(dims) -> tuple:
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx, 4, 3)


def site_axis(mu: int) -> int:
    """Array axis (counted from the end of a spinor field) of direction mu."""
    return -6 + (3 - mu)


def coordinates(dims):
    """Arrays x, y, z, t of shape (T, Lz, Ly, Lx) giving each site's coordinates."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return x, y, z, t


def lexicographic_index(x, y, z, t, dims):
    """i = x + Lx*(y + Ly*(z + Lz*t))."""
    lx, ly, lz, _ = dims
    return x + lx * (y + ly * (z + lz * t))


def parity(x, y, z, t):
    """Even-odd parity (x + y + z + t) mod 2."""
    return (x + y + z + t) & 1


# --- gamma matrices (DeGrand-Rossi chiral basis) ---------------------------------

def gammas() -> np.ndarray:
    """gamma_1..gamma_4 as complex128[4, 4, 4] (index 0..3 <-> gamma_1..gamma_4)."""
    i = 1j
    g1 = np.array([[0, 0, 0, i], [0, 0, i, 0], [0, -i, 0, 0], [-i, 0, 0, 0]], dtype=np.complex128)
    g2 = np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=np.complex128)
    g3 = np.array([[0, 0, i, 0], [0, 0, 0, -i], [-i, 0, 0, 0], [0, i, 0, 0]], dtype=np.complex128)
    g4 = np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=np.complex128)
    return np.stack([g1, g2, g3, g4])


def gamma5() -> np.ndarray:
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


# Order of the 16-element Gamma basis used for every loop output.
GAMMA_NAMES = (
    "1",
    "g1", "g2", "g3", "g4",
    "g5",
    "g5g1", "g5g2", "g5g3", "g5g4",
    "g1g2", "g1g3", "g1g4", "g2g3", "g2g4", "g3g4",
)


def gamma_basis() -> np.ndarray:
    """The 16 Gamma matrices in the order of GAMMA_NAMES, complex128[16, 4, 4]."""
    g = gammas()
    g5 = gamma5()
    out = [np.eye(4, dtype=np.complex128)]
    out += [g[m] for m in range(4)]
    out += [g5]
    out += [g5 @ g[m] for m in range(4)]
    for a in range(4):
        for b in range(a + 1, 4):
            out.append(g[a] @ g[b])
    return np.stack(out)
