"""Complex Z2 noise sources and dilution (oracle; test infrastructure).

Sec. 2 of the paper: the stochastic loops use complex Z2 noise for the source
vectors together with dilution (partitioning) of the source index set: colour
dilution (x3 inversions), full spin dilution (x4), an even-odd spatial
partitioning (x2), a cubic spatial partitioning (x8: one class per vertex of
the elementary 3-cube, repeated over the lattice) and time dilution, which by
translation invariance costs no extra inversions.

Readings (the paper gives the factors only):

* noise vector n has entries xi_n(x, alpha, a) = (s_re + i s_im) / sqrt(2), the
  magnitude 1/sqrt(2) being the double nearest to it (sqrt(0.5)), with
  signs s = +-1 drawn by Philox4x64-10 under key (seed, 0) and counter
  (i >> 2, n, 0, 0), i the lexicographic site index: 64-bit word (i & 3) of the
  output block belongs to site i; component c = 3*alpha + a takes its real sign
  from bit 2c and its imaginary sign from bit 2c+1 (bit set -> sign -1);
* dilution multiplies one noise vector by the indicator P_k of class k, so the
  diluted sources of one noise vector sum back to it;  the classes combine as a
  mixed-radix index k = ((k_spin*C + k_colour)*E + k_eo)*Q + k_cubic with each
  absent factor of size 1 (C = 3, E = 2, Q = 8 when present);
  spin class = alpha, colour class = a, even-odd class = (x+y+z+t) & 1, cubic
  class = (x&1) + 2(y&1) + 4(z&1);
* time dilution keeps only timeslice t0(n) = t0 if t0 >= 0, else n mod T (the
  source timeslice translated with the noise index);
* diluted right-hand side number r = (n - noise_first) * K + k.
"""

from __future__ import annotations

import numpy as np

from .lattice import coordinates, lexicographic_index, parity, spinor_shape
from .philox import philox4x64

SPIN, COLOUR, EVENODD, CUBIC, TIME = 1, 2, 4, 8, 16


def dilution_sizes(dilution: int):
    """(spin, colour, even-odd, cubic) class counts for a dilution bitmask."""
    return (
        4 if dilution & SPIN else 1,
        3 if dilution & COLOUR else 1,
        2 if dilution & EVENODD else 1,
        8 if dilution & CUBIC else 1,
    )


def n_classes(dilution: int) -> int:
    s, c, e, q = dilution_sizes(dilution)
    return s * c * e * q


def z2_noise(dims, seed: int, n: int) -> np.ndarray:
    """The undiluted complex Z2 vector xi_n, complex128[T, Lz, Ly, Lx, 4, 3]."""
    x, y, z, t = coordinates(dims)
    site = lexicographic_index(x, y, z, t, dims).astype(np.uint64)
    counter = np.zeros(site.shape + (4,), dtype=np.uint64)
    counter[..., 0] = site >> np.uint64(2)
    counter[..., 1] = np.uint64(n)
    key = np.array([seed & (2**64 - 1), 0], dtype=np.uint64)
    block = philox4x64(counter, key)
    word = np.take_along_axis(block, (site & np.uint64(3)).astype(np.int64)[..., None], axis=-1)[..., 0]
    out = np.empty(site.shape + (4, 3), dtype=np.complex128)
    for alpha in range(4):
        for a in range(3):
            c = 3 * alpha + a
            bre = (word >> np.uint64(2 * c)) & np.uint64(1)
            bim = (word >> np.uint64(2 * c + 1)) & np.uint64(1)
            sre = 1.0 - 2.0 * bre.astype(np.float64)
            sim = 1.0 - 2.0 * bim.astype(np.float64)
            out[..., alpha, a] = (sre + 1j * sim) * np.sqrt(0.5)
    return out


def class_mask(dims, dilution: int, k: int, t0: int | None) -> np.ndarray:
    """Boolean mask [T, Lz, Ly, Lx, 4, 3] of dilution class k (time: slice t0)."""
    ns, nc, ne, nq = dilution_sizes(dilution)
    k_q = k % nq
    k_e = (k // nq) % ne
    k_c = (k // (nq * ne)) % nc
    k_s = k // (nq * ne * nc)
    x, y, z, t = coordinates(dims)
    site_ok = np.ones(x.shape, dtype=bool)
    if dilution & EVENODD:
        site_ok &= parity(x, y, z, t) == k_e
    if dilution & CUBIC:
        site_ok &= ((x & 1) + 2 * (y & 1) + 4 * (z & 1)) == k_q
    if dilution & TIME:
        site_ok &= t == t0
    spin_ok = np.ones(4, dtype=bool) if not dilution & SPIN else (np.arange(4) == k_s)
    col_ok = np.ones(3, dtype=bool) if not dilution & COLOUR else (np.arange(3) == k_c)
    return site_ok[..., None, None] & spin_ok[:, None] & col_ok[None, :]


def source_timeslice(n: int, t0: int, lt: int) -> int:
    return t0 if t0 >= 0 else n % lt


def make_sources(dims, seed: int, noise_first: int, n_noise: int, dilution: int, t0: int = 0):
    """All diluted sources eta_{n,k} for n in [noise_first, noise_first + n_noise).

    Returns complex128[n_noise * K, T, Lz, Ly, Lx, 4, 3] in right-hand-side order.
    """
    lt = dims[3]
    kk = n_classes(dilution)
    out = np.zeros((n_noise * kk,) + spinor_shape(dims), dtype=np.complex128)
    for j in range(n_noise):
        n = noise_first + j
        xi = z2_noise(dims, seed, n)
        tn = source_timeslice(n, t0, lt) if dilution & TIME else None
        for k in range(kk):
            out[j * kk + k] = np.where(class_mask(dims, dilution, k, tn), xi, 0)
    return out


def point_sources(dims, first: int, n: int) -> np.ndarray:
    """Unit sources e_{y,alpha,a} with source index s = 12*y + 3*alpha + a."""
    lx, ly, lz, lt = dims
    out = np.zeros((n,) + spinor_shape(dims), dtype=np.complex128)
    flat = out.reshape(n, -1)
    for j in range(n):
        flat[j, first + j] = 1.0
    return out
