"""Pins for the oracle's Philox generator, complex Z2 noise and dilution (CPU)."""

import numpy as np
import pytest

from oracle import noise, philox


def _numpy_philox_blocks(key, counter_start, n_blocks):
    """Reference blocks from numpy's own Philox4x64-10 bit generator.

    numpy increments its 256-bit counter before producing each block, so a
    generator started at counter C - 1 emits philox(C), philox(C + 1), ...
    """
    c_int = sum(int(w) << (64 * i) for i, w in enumerate(counter_start))
    bg = np.random.Philox(key=[int(key[0]), int(key[1])], counter=(c_int - 1) % (1 << 256))
    return bg.random_raw(4 * n_blocks).reshape(n_blocks, 4)


@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (0, 0, 0, 0)),
    ((12345, 0), (7, 3, 0, 0)),
    ((2**64 - 1, 2**63 + 5), (2**64 - 3, 2**64 - 1, 17, 2**62)),
])
def test_philox_matches_numpy(key, ctr):
    n = 9
    ref = _numpy_philox_blocks(key, ctr, n)
    c_int = sum(int(w) << (64 * i) for i, w in enumerate(ctr))
    ctrs = []
    for j in range(n):
        v = (c_int + j) % (1 << 256)
        ctrs.append([(v >> (64 * i)) & (2**64 - 1) for i in range(4)])
    got = philox.philox4x64(np.array(ctrs, dtype=np.uint64), np.array(key, dtype=np.uint64))
    assert np.array_equal(got, ref)


def test_z2_values_and_bit_map():
    dims = (4, 2, 2, 4)
    xi = noise.z2_noise(dims, seed=99, n=5)
    assert np.allclose(np.abs(xi.real), 1 / np.sqrt(2)) and np.allclose(np.abs(xi.imag), 1 / np.sqrt(2))
    # site 6 lives in block 1 (counter (1, 5, 0, 0)), word 2
    block = philox.philox4x64(np.array([1, 5, 0, 0], dtype=np.uint64), np.array([99, 0], dtype=np.uint64))
    w = int(block[2])
    flat = xi.reshape(-1, 12)
    for c in range(12):
        re = -1 if (w >> (2 * c)) & 1 else 1
        im = -1 if (w >> (2 * c + 1)) & 1 else 1
        assert flat[6, c] == pytest.approx((re + 1j * im) / np.sqrt(2))


def test_z2_second_moment():
    """E[xi xi^dagger] = 1: off-diagonal averages vanish like 1/sqrt(N)."""
    dims = (4, 4, 4, 4)
    xs = np.stack([noise.z2_noise(dims, 3, n).reshape(-1) for n in range(64)])
    m = (xs[:, :, None] * xs[:, None, :200].conj()).mean(axis=0)[:200]
    assert np.allclose(np.diag(m), 1.0)
    off = m - np.diag(np.diag(m))
    assert np.abs(off).max() < 6 / np.sqrt(64)


@pytest.mark.parametrize("dil", [
    0, noise.SPIN, noise.COLOUR, noise.SPIN | noise.COLOUR,
    noise.SPIN | noise.COLOUR | noise.EVENODD, noise.CUBIC, noise.COLOUR | noise.CUBIC | noise.TIME,
    noise.SPIN | noise.COLOUR | noise.EVENODD | noise.TIME,
])
def test_dilution_partitions_the_noise(dil):
    dims = (4, 4, 2, 4)
    kk = noise.n_classes(dil)
    srcs = noise.make_sources(dims, seed=5, noise_first=3, n_noise=2, dilution=dil, t0=-1)
    assert srcs.shape[0] == 2 * kk
    for j in range(2):
        n = 3 + j
        xi = noise.z2_noise(dims, 5, n)
        block = srcs[j * kk:(j + 1) * kk]
        nz = (block != 0).sum(axis=0)
        assert nz.max() <= 1  # classes are disjoint
        total = block.sum(axis=0)
        if dil & noise.TIME:
            tn = n % dims[3]
            assert np.array_equal(total[tn], xi[tn])
            assert np.all(np.delete(total, tn, axis=0) == 0)
        else:
            assert np.array_equal(total, xi)


def test_dilution_class_membership():
    dims = (4, 4, 4, 2)
    dil = noise.SPIN | noise.COLOUR | noise.EVENODD | noise.CUBIC
    assert noise.n_classes(dil) == 4 * 3 * 2 * 8
    k = ((2 * 3 + 1) * 2 + 1) * 8 + 5  # spin 2, colour 1, odd sites, cubic class 5
    m = noise.class_mask(dims, dil, k, None)
    lx, ly, lz, lt = dims
    for t in range(lt):
        for z in range(lz):
            for y in range(ly):
                for x in range(lx):
                    for s in range(4):
                        for a in range(3):
                            want = (s == 2 and a == 1 and (x + y + z + t) % 2 == 1
                                    and (x % 2) + 2 * (y % 2) + 4 * (z % 2) == 5)
                            assert m[t, z, y, x, s, a] == want


def test_point_sources():
    dims = (2, 2, 2, 2)
    p = noise.point_sources(dims, first=37, n=3)
    flat = p.reshape(3, -1)
    for j in range(3):
        assert flat[j].sum() == 1 and flat[j, 37 + j] == 1
