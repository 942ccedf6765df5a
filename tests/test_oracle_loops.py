"""Pins for the oracle's loops, smearing, TSM combination and gradients (CPU)."""

import numpy as np
import pytest

import synthetic
from oracle import lattice, loops, noise, smear, wilson

TBC = -1.0


def _gauge_transform_links(u, g):
    out = np.empty_like(u)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=lattice.site_axis(mu))
        out[..., mu, :, :] = g @ u[..., mu, :, :] @ g_fwd.conj().swapaxes(-1, -2)
    return out


@pytest.fixture(scope="module")
def small():
    dims = (2, 2, 2, 4)
    u = synthetic.gauge_field(dims, eps=0.5, seed=4)
    kappa = 0.12
    m = wilson.dense_matrix(u, kappa, TBC)
    return dims, u, kappa, m, np.linalg.inv(m)


def test_exact_loops_from_point_solves_equal_dense(small):
    dims, u, kappa, m, minv = small
    v = lattice.volume(dims)
    idx = np.arange(12 * v)
    phi = minv.T.reshape((12 * v,) + lattice.spinor_shape(dims))  # column s of M^-1
    lo_pts = loops.point_diagonal_loops(dims, idx, phi)
    lo_dense = loops.exact_loops_dense(u, kappa, TBC)
    assert np.allclose(lo_pts, lo_dense, atol=1e-13)
    # brute force over sites for one Gamma and one timeslice
    gam = lattice.gamma_basis()[11]
    blocks = minv.reshape(v, 12, v, 12)
    t = 2
    sites = range(t * v // dims[3], (t + 1) * v // dims[3])
    ref = sum(np.trace(np.kron(gam, np.eye(3)) @ blocks[x, :, x, :]) for x in sites)
    assert abs(lo_dense[11, t] - ref) < 1e-13


def test_point_source_contraction_reproduces_exact(small):
    """With eta = e_s for every s (full dilution), sum_s eta^dag Gamma phi = exact loops."""
    dims, u, kappa, m, minv = small
    v = lattice.volume(dims)
    eta = noise.point_sources(dims, 0, 12 * v)
    phi = (minv @ eta.reshape(12 * v, -1).T).T.reshape(eta.shape)
    est = loops.stochastic_loops(eta, phi).sum(axis=0)
    assert np.allclose(est, loops.exact_loops_dense(u, kappa, TBC), atol=1e-13)


def test_gamma5_hermiticity_of_loops():
    """L_1, L_g5, L_g5gmu real; L_gmu, L_gmugnu imaginary (gamma5 M gamma5 = M^dag)."""
    dims = (4, 4, 4, 4)
    u = synthetic.gauge_field(dims, eps=0.3, seed=1)
    lo = loops.exact_loops_dense(u, 0.10, TBC)
    scale = np.abs(lo).max()
    real_idx = [0, 5, 6, 7, 8, 9]
    imag_idx = [1, 2, 3, 4, 10, 11, 12, 13, 14, 15]
    assert np.abs(lo[real_idx].imag).max() < 1e-14 * scale
    assert np.abs(lo[imag_idx].real).max() < 1e-14 * scale


def test_gauge_invariance_of_exact_loops():
    dims = (2, 2, 4, 4)
    u = synthetic.gauge_field(dims, eps=0.45, seed=8)
    g = synthetic.random_gauge_transform(dims, seed=9)
    a = loops.exact_loops_dense(u, 0.13, TBC)
    b = loops.exact_loops_dense(_gauge_transform_links(u, g), 0.13, TBC)
    assert np.abs(a - b).max() < 1e-12


def test_stochastic_estimator_is_unbiased(small):
    dims, u, kappa, m, minv = small
    v = lattice.volume(dims)
    nn = 400
    eta = np.stack([noise.z2_noise(dims, 17, n) for n in range(nn)])
    phi = (minv @ eta.reshape(nn, -1).T).T.reshape(eta.shape)
    est = loops.stochastic_loops(eta, phi)
    mean = est.mean(axis=0)
    err = est.std(axis=0) / np.sqrt(nn)
    exact = loops.exact_loops_dense(u, kappa, TBC)
    z = np.abs(mean - exact) / np.maximum(err, 1e-12)
    assert np.median(z) < 1.5 and z.max() < 5.5
    # Gamma = 1 on the diagonal carries no noise from the diagonal itself
    assert v > 0


def test_smearing_free_field_plane_wave():
    """U = 1: K e^{ipx} = [(1 + 2 alpha sum_j cos p_j)/(1 + 6 alpha)]^n e^{ipx}."""
    dims = (4, 6, 8, 2)
    u1 = synthetic.unit_gauge(dims)
    x, y, z, t = lattice.coordinates(dims)
    p = (2 * np.pi / 4, 2 * np.pi * 2 / 6, 2 * np.pi * 3 / 8)
    psi = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + 0.7 * t))[..., None, None] * np.ones((4, 3))
    alpha, n = 4.0, 7
    fac = ((1 + 2 * alpha * sum(np.cos(q) for q in p)) / (1 + 6 * alpha)) ** n
    assert np.allclose(smear.smear(u1, psi, alpha, n), fac * psi, atol=1e-13)


def test_smearing_hermitian_and_covariant():
    dims = (4, 4, 4, 2)
    u = synthetic.gauge_field(dims, eps=0.45, seed=3)
    a = synthetic.random_spinor(dims, 1)
    b = synthetic.random_spinor(dims, 2)
    ka = smear.smear(u, a, 4.0, 5)
    kb = smear.smear(u, b, 4.0, 5)
    assert abs(np.vdot(a, kb) - np.vdot(ka, b)) < 1e-12 * abs(np.vdot(a, kb))
    g = synthetic.random_gauge_transform(dims, 5)
    ug = _gauge_transform_links(u, g)
    lhs = smear.smear(ug, a @ g.swapaxes(-1, -2), 4.0, 5)
    assert np.abs(lhs - ka @ g.swapaxes(-1, -2)).max() < 1e-12
    # time slices do not mix
    a0 = np.zeros_like(a)
    a0[1] = a[1]
    assert np.all(smear.smear(u, a0, 4.0, 3)[0] == 0)


def test_smeared_stochastic_estimator_matches_exact_smeared(small):
    """Point-source (full-dilution) estimator with K eta, K phi equals Tr[Gamma K M^-1 K]."""
    dims, u, kappa, m, minv = small
    v = lattice.volume(dims)
    eta = noise.point_sources(dims, 0, 12 * v)
    phi = (minv @ eta.reshape(12 * v, -1).T).T.reshape(eta.shape)
    est = loops.smeared_loops(u, eta, phi, 2.0, 3).sum(axis=0)
    ref = loops.exact_smeared_loops_dense(u, kappa, 2.0, 3, TBC)
    assert np.allclose(est, ref, atol=1e-12)


def test_tsm_combination():
    rng = np.random.default_rng(0)
    n_lp, n_hp, lt = 50, 10, 4
    lp = rng.standard_normal((n_lp, 16, lt)) + 1j * rng.standard_normal((n_lp, 16, lt))
    hp = rng.standard_normal((n_hp, 16, lt)) + 1j * rng.standard_normal((n_hp, 16, lt))
    # f_HP == f_LP on the HP ensemble: the correction vanishes exactly
    mean, var = loops.tsm_estimate(lp, hp, hp.copy())
    assert np.array_equal(mean, lp.mean(axis=0))
    # brute-force mean and variance of the mean
    lp_on_hp = hp + 0.1 * rng.standard_normal(hp.shape)
    mean, var = loops.tsm_estimate(lp, hp, lp_on_hp)
    d = hp - lp_on_hp
    assert np.allclose(mean, lp.mean(0) + d.mean(0))
    v_ref = np.var(lp, axis=0, ddof=1) / n_lp + np.var(d, axis=0, ddof=1) / n_hp
    assert np.allclose(var, v_ref)
    # time coverage: only covered timeslices enter
    cover = np.zeros((n_lp, lt), dtype=bool)
    cover[np.arange(n_lp), np.arange(n_lp) % lt] = True
    m2, _ = loops.tsm_estimate(lp, hp, lp_on_hp, lp_cover=cover)
    assert np.allclose(m2[:, 1], lp[1::lt, :, 1].mean(0) + d[:, :, 1].mean(0))


def test_tsm_is_unbiased_for_a_crude_low_precision_map(small):
    """TSM with a deliberately bad deterministic f_LP still averages to the exact loops."""
    dims, u, kappa, m, minv = small
    v = lattice.volume(dims)

    def f_lp(eta):  # truncated hopping series: a fixed, inaccurate map
        out = eta.copy()
        term = eta.copy()
        for _ in range(3):
            term = kappa * wilson.hop(u, term, TBC)
            out = out + term
        return out

    def f_hp(eta):
        return (minv @ eta.reshape(len(eta), -1).T).T.reshape(eta.shape)

    n_lp, n_hp = 600, 300
    e_lp = np.stack([noise.z2_noise(dims, 1, n) for n in range(n_lp)])
    e_hp = np.stack([noise.z2_noise(dims, 1, n) for n in range(n_lp, n_lp + n_hp)])
    lp = loops.stochastic_loops(e_lp, f_lp(e_lp))
    hp = loops.stochastic_loops(e_hp, f_hp(e_hp))
    lph = loops.stochastic_loops(e_hp, f_lp(e_hp))
    mean, var = loops.tsm_estimate(lp, hp, lph)
    exact = loops.exact_loops_dense(u, kappa, TBC)
    z = np.abs(mean - exact) / np.sqrt(np.maximum(var, 1e-24))
    assert np.median(z) < 1.5 and z.max() < 5.5
    assert v > 0


def test_loop_gradients_match_torch_autograd():
    """Adjoint-based gradients vs torch autograd through a dense solve (2x2x2x4)."""
    torch = pytest.importorskip("torch")
    dims = (2, 2, 2, 4)
    u = synthetic.gauge_field(dims, eps=0.5, seed=6)
    kappa = 0.11
    gidx = 5  # gamma_5
    eta = noise.z2_noise(dims, 2, 0)
    v = lattice.volume(dims)
    lt = dims[3]
    d_dense = (np.eye(12 * v) - wilson.dense_matrix(u, 1.0, TBC))  # D = 1 - M(kappa=1)
    gam = np.kron(lattice.gamma_basis()[gidx], np.eye(3))
    D = torch.tensor(d_dense)
    G = torch.tensor(np.kron(np.eye(v), gam))
    e = torch.tensor(eta.reshape(-1), requires_grad=True)
    k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    M = torch.eye(12 * v, dtype=torch.complex128) - k * D
    phi = torch.linalg.solve(M, e)
    prod = (e.conj() * (G @ phi)).reshape(lt, -1).sum(dim=1)  # L(t)
    c = torch.tensor(np.random.default_rng(1).standard_normal(lt) + 1j * np.random.default_rng(2).standard_normal(lt))
    L = prod.detach().requires_grad_(True)
    loss_fn = lambda z: (c.conj() * z).real.sum() + 0.3 * (z.abs() ** 2).sum()  # noqa: E731
    loss_fn(L).backward()
    g = L.grad.numpy().copy()
    loss_fn(prod).backward()
    ge, gk = loops.loop_gradients(u, kappa, eta, gidx, g, TBC)
    assert np.allclose(ge.reshape(-1), e.grad.numpy(), atol=1e-10)
    assert abs(gk - k.grad.item()) < 1e-9 * max(1.0, abs(gk))


def test_dilution_sigma2_pins():
    """The dilution-study statistic: (a) with the exact loops replaced by the sample means it is
    numpy's variance (mean |x - mean|^2) of the estimates, weighted by the vectors per timeslice;
    (b) offsets c_n common to every Gamma give sigma2 = mean |c_n|^2."""
    rng = np.random.default_rng(7)
    n, T = 12, 4
    L = rng.standard_normal((n, 16, T)) + 1j * rng.standard_normal((n, 16, T))
    t_of = [i % T for i in range(n)]
    means = np.stack([L[[i for i in range(n) if t_of[i] == t], :, t].mean(0) for t in range(T)], axis=-1)
    got = loops.dilution_sigma2(L, means, t_of)
    ref = sum(np.var(L[[i for i in range(n) if t_of[i] == t], :, t], axis=0) * t_of.count(t) for t in range(T)) / n
    assert np.allclose(got, ref, rtol=1e-13)
    assert np.allclose(loops.dilution_sigma2(L, L.mean(0), None), np.var(L, axis=0).mean(-1), rtol=1e-13)
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    exact = rng.standard_normal((16, T)) + 1j * rng.standard_normal((16, T))
    shifted = exact[None] + c[:, None, None]
    assert np.allclose(loops.dilution_sigma2(shifted, exact, t_of), np.mean(np.abs(c) ** 2), rtol=1e-13)


def test_full_dilution_has_no_stochastic_error():
    """On a 2x2x2x4 lattice, spin x colour x cubic x time dilution puts every class on one site,
    spin and colour: each noise vector's estimate is the exact loop on its timeslice, so the
    dilution-study statistic vanishes (to solver tolerance)."""
    dims, kappa = (2, 2, 2, 4), 0.11
    U = synthetic.gauge_field(dims, eps=0.45, seed=8)
    exact = loops.exact_loops_dense(U, kappa, -1.0)
    dil = noise.SPIN | noise.COLOUR | noise.CUBIC | noise.TIME
    per = []
    for n in range(3):
        eta = noise.make_sources(dims, 5, n, 1, dil, t0=-1)
        phi = np.stack([wilson.solve(U, e, kappa, -1.0, tol=1e-13)[0] for e in eta])
        per.append(loops.stochastic_loops(eta, phi).sum(0))
    sig = loops.dilution_sigma2(np.array(per), exact, [n % 4 for n in range(3)])
    assert sig.max() < 1e-20 * np.abs(exact).max() ** 2 + 1e-22
