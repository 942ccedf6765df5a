"""Philox4x64-10 counter-based generator (oracle; test infrastructure).

The paper draws complex Z2 noise (Sec. 2) without naming a generator.  Both the
CUDA path and this oracle use Philox4x64-10 as published by Salmon, Moraes,
Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): a
10-round Feistel-like bijection of a 256-bit counter under a 128-bit key.

One round maps counter (c0, c1, c2, c3) under key (k0, k1) to

    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))

where hi/lo are the upper/lower 64 bits of the 128-bit product; between rounds
the key is bumped by the Weyl constants (k0 += W0, k1 += W1 mod 2^64).

This is an independent restatement in numpy uint64 arithmetic; the test suite
pins it against numpy's own Philox bit generator.
"""

from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def mulhilo64(a, b):
    """(hi, lo) 64-bit halves of the 128-bit product a*b, elementwise on uint64."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a0, a1 = a & _LO32, a >> _S32
    b0, b1 = b & _LO32, b >> _S32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> _S32) + (p01 & _LO32) + (p10 & _LO32)
    lo = a * b  # wraps mod 2^64
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64(counter, key, rounds: int = 10):
    """Apply Philox4x64-R to counters.

    counter: uint64 array [..., 4]; key: uint64 array [..., 2] (broadcastable).
    Returns uint64 array [..., 4].
    """
    with np.errstate(over="ignore"):
        c = np.asarray(counter, dtype=np.uint64)
        k = np.asarray(key, dtype=np.uint64)
        shape = np.broadcast_shapes(c.shape[:-1], k.shape[:-1])
        c = np.broadcast_to(c, shape + (4,)).copy()
        k0 = np.broadcast_to(k[..., 0], shape).copy()
        k1 = np.broadcast_to(k[..., 1], shape).copy()
        for r in range(rounds):
            if r > 0:
                k0 = k0 + W0
                k1 = k1 + W1
            hi0, lo0 = mulhilo64(M0, c[..., 0])
            hi1, lo1 = mulhilo64(M1, c[..., 2])
            c = np.stack([hi1 ^ c[..., 1] ^ k0, lo1, hi0 ^ c[..., 3] ^ k1, lo0], axis=-1)
        return c
