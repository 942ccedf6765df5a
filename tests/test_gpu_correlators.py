"""Momentum-projected loops and two-point functions vs the oracle (GPU)."""

import numpy as np
import pytest

import synthetic
from oracle import correlators, lattice, smear, wilson

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

G16 = lattice.gamma_basis()
MOMENTA = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 1), (0, -1, -1), (2, 1, -1), (-2, -1, 1)]


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_momentum_loops_match_oracle(lib):
    dims = (4, 4, 2, 8)
    U = synthetic.gauge_field(dims, eps=0.45, seed=21)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(0.12)
    eta = synthetic.random_spinor(dims, seed=22, n=5)
    phi = synthetic.random_spinor(dims, seed=23, n=5)
    got = c.trace_loops_mom(to_gpu(eta), to_gpu(phi), MOMENTA, lib.SINK_LOCAL | lib.SINK_SMEARED, smear=(3.0, 4))
    assert got.shape == (5, 2, len(MOMENTA), 16, 8)
    ref_l = correlators.momentum_loops(eta, phi, MOMENTA, G16)
    se = np.stack([smear.smear(U, e, 3.0, 4) for e in eta])
    sf = np.stack([smear.smear(U, f, 3.0, 4) for f in phi])
    ref_s = correlators.momentum_loops(se, sf, MOMENTA, G16)
    assert np.abs(got[:, 0] - ref_l).max() < 1e-12 * np.abs(ref_l).max()
    assert np.abs(got[:, 1] - ref_s).max() < 1e-12 * np.abs(ref_s).max()
    # zero momentum is the ordinary loop
    plain = c.trace_loops(to_gpu(eta), to_gpu(phi), lib.SINK_LOCAL)
    assert np.abs(got[:, 0, 0] - plain[:, 0]).max() < 1e-12 * np.abs(plain).max()
    c.close()


def test_momentum_loops_per_rhs_timeslice_and_groups(lib):
    dims = (4, 2, 4, 4)
    c = lib.Context(dims)
    c.load_gauge(synthetic.gauge_field(dims, eps=0.45, seed=24))
    eta = synthetic.random_spinor(dims, seed=25, n=6)
    phi = synthetic.random_spinor(dims, seed=26, n=6)
    t_of = [1, 1, 3, 3, 0, 0]
    got = c.trace_loops_mom(to_gpu(eta), to_gpu(phi), MOMENTA[:3], lib.SINK_LOCAL, t_of_rhs=t_of, group=2)
    ref = correlators.momentum_loops(eta, phi, MOMENTA[:3], G16)  # [6][Q][16][T]
    for g in range(3):
        want = np.zeros((3, 16, 4), complex)
        t0 = t_of[2 * g]
        want[:, :, t0] = ref[2 * g, :, :, t0] + ref[2 * g + 1, :, :, t0]
        assert np.abs(got[g, 0] - want).max() < 1e-12 * np.abs(ref).max()
    c.close()


def block_error(got, ref):
    """Per (p, Gamma_A, Gamma_B): ||got - ref|| / max(||ref||, 1e-6 ||C_pion(p = 0)||) over the timeslices."""
    floor = 1e-6 * np.linalg.norm(ref[0, 5, 5])
    num = np.linalg.norm(got - ref, axis=-1)
    return num / np.maximum(np.linalg.norm(ref, axis=-1), floor)


def test_meson_correlators_match_oracle(lib):
    """Point source at (1, 2, 0, 5): GPU solve (FP32 inner, FP64 defect correction to 1e-13) and
    contraction vs the oracle's contraction of the dense-inverse columns, compared per momentum
    and per (Gamma_A, Gamma_B) pair, each against its own norm."""
    dims, kappa, src = (4, 4, 2, 8), 0.12, (1, 2, 0, 5)
    U = synthetic.gauge_field(dims, eps=0.45, seed=27)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    i = src[0] + dims[0] * (src[1] + dims[1] * (src[2] + dims[2] * src[3]))
    b = c.make_point_sources(12 * i, 12)
    prop, st = c.solve(b, lib.Params(tol=1e-13, precision=1, batch=16))
    got = c.meson_correlators(prop, src, MOMENTA[:4])
    minv = np.linalg.inv(wilson.dense_matrix(U, kappa, -1.0, dims))
    lx, ly, lz, lt = dims
    exact = minv[:, 12 * i:12 * i + 12].T.reshape(12, lt, lz, ly, lx, 4, 3)
    ref = correlators.connected(exact, src, MOMENTA[:4], G16)
    err = block_error(got, ref)
    print("connected: max per-(p,A,B) error %.3e" % err.max())
    assert err.max() < 1e-9
    pion = got[0, 5, 5]
    assert np.all(pion.real < 0) and np.abs(pion.imag).max() < 1e-10 * np.abs(pion).max()
    c.close()


def test_disconnected_matches_oracle_pairs(lib):
    """Per-noise loops drawn on the host; the GPU pair estimator equals the oracle's brute force."""
    dims = (4, 4, 2, 6)
    c = lib.Context(dims)
    rng = np.random.default_rng(28)
    n, Q, T = 5, 3, dims[3]
    moms = [(0, 0, 0), (1, 0, 0), (-1, 0, 0)]
    L = rng.standard_normal((n, Q, 16, T)) + 1j * rng.standard_normal((n, Q, 16, T))
    cover = rng.random((n, T)) < 0.6
    cover[:, 0] = True
    got = c.disconnected(L, moms, cover)
    ref = correlators.disconnected_pairs(L, cover, [0, 2, 1], spatial_volume=32)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
    full = c.disconnected(L, moms)
    assert np.abs(full - correlators.disconnected_pairs(L, None, [0, 2, 1], 32)).max() < 1e-13 * np.abs(full).max()
    with pytest.raises(lib.DlError):
        c.disconnected(L[:, :2], moms[:2])  # -p of (1, 0, 0) missing
    c.close()
