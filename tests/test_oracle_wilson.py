"""Pins for the oracle's Wilson operator and solver (CPU).

Each check comes from outside the oracle: the momentum-space form of the free
Wilson operator, a dense LAPACK solve, gamma5-hermiticity, gauge covariance and
the hopping expansion of M^{-1} (whose kappa^4 term is a sum over plaquettes).
"""

import itertools

import numpy as np
import pytest

import synthetic
from oracle import lattice, wilson

TBC = -1.0


def _plane_wave(dims, n_mom, spin_colour):
    """e^{i p.x} u with p_i = 2 pi n_i / L_i and antiperiodic p_4 = (2 n_4 + 1) pi / T."""
    lx, ly, lz, lt = dims
    x, y, z, t = lattice.coordinates(dims)
    p = np.array([2 * np.pi * n_mom[0] / lx, 2 * np.pi * n_mom[1] / ly,
                  2 * np.pi * n_mom[2] / lz, (2 * n_mom[3] + 1) * np.pi / lt])
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return phase[..., None, None] * spin_colour, p


def test_free_hop_on_plane_wave():
    """D e^{ipx} u = [2 sum cos p_mu - 2i sum gamma_mu sin p_mu] e^{ipx} u."""
    dims = (4, 6, 2, 8)
    u1 = synthetic.unit_gauge(dims)
    rng = np.random.default_rng(0)
    sc = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    g = lattice.gammas()
    for n_mom in [(0, 0, 0, 0), (1, 2, 1, 3), (3, 5, 0, 7)]:
        psi, p = _plane_wave(dims, n_mom, sc)
        dp = 2 * np.cos(p).sum() * np.eye(4) - 2j * sum(g[m] * np.sin(p[m]) for m in range(4))
        expect = np.einsum("sr,...ra->...sa", dp, psi)
        assert np.allclose(wilson.hop(u1, psi, TBC), expect, atol=1e-12)


def _free_trace_closed_form(dims, kappa):
    """(12/V) sum_p A/(A^2 + B^2), A = 1 - 2 kappa sum cos p, B^2 = 4 kappa^2 sum sin^2 p."""
    lx, ly, lz, lt = dims
    ps = [2 * np.pi * np.arange(lx) / lx, 2 * np.pi * np.arange(ly) / ly,
          2 * np.pi * np.arange(lz) / lz, (2 * np.arange(lt) + 1) * np.pi / lt]
    P = np.meshgrid(*ps, indexing="ij")
    a = 1 - 2 * kappa * sum(np.cos(q) for q in P)
    b2 = 4 * kappa ** 2 * sum(np.sin(q) ** 2 for q in P)
    return 12.0 / lattice.volume(dims) * np.sum(a / (a * a + b2))


def test_free_field_closed_form_trace():
    """Exact free-field loops: Tr M^{-1}(x,x) from the momentum sum; other Gamma vanish."""
    from oracle import loops
    dims = (4, 4, 4, 4)
    kappa = 0.10
    lo = loops.exact_loops_dense(synthetic.unit_gauge(dims), kappa, TBC)
    per_site = _free_trace_closed_form(dims, kappa)
    assert abs(per_site - 11.86554754963829) < 1e-12
    sites_per_t = 64
    assert np.allclose(lo[0], per_site * sites_per_t, rtol=1e-13)
    assert np.abs(lo[1:]).max() < 1e-12


def test_bicgstab_matches_dense_lapack_solve():
    dims = (2, 2, 2, 2)
    u = synthetic.gauge_field(dims, eps=0.5, seed=7)
    kappa = 0.12
    b = synthetic.random_spinor(dims, seed=3)
    x, info = wilson.solve(u, b, kappa, TBC, tol=1e-13)
    m = wilson.dense_matrix(u, kappa, TBC)
    x_ref = np.linalg.solve(m, b.ravel())
    assert info["converged"]
    assert np.linalg.norm(x.ravel() - x_ref) / np.linalg.norm(x_ref) < 1e-11


def test_gamma5_hermiticity_dense():
    dims = (2, 2, 2, 2)
    u = synthetic.gauge_field(dims, eps=0.7, seed=5)
    m = wilson.dense_matrix(u, 0.13, TBC)
    g5 = np.kron(np.eye(lattice.volume(dims)), np.kron(lattice.gamma5(), np.eye(3)))
    assert np.abs(g5 @ m @ g5 - m.conj().T).max() < 1e-15


def test_adjoint_inner_product():
    dims = (4, 2, 2, 4)
    u = synthetic.gauge_field(dims, eps=0.45, seed=2)
    a = synthetic.random_spinor(dims, seed=1)
    b = synthetic.random_spinor(dims, seed=2)
    lhs = np.vdot(a.ravel(), wilson.apply_m(u, b, 0.14, TBC).ravel())
    rhs = np.vdot(wilson.apply_mdag(u, a, 0.14, TBC).ravel(), b.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _gauge_transform_links(u, g):
    """U_mu(x) -> g(x) U_mu(x) g(x + mu)^dagger."""
    out = np.empty_like(u)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=lattice.site_axis(mu))
        out[..., mu, :, :] = g @ u[..., mu, :, :] @ g_fwd.conj().swapaxes(-1, -2)
    return out


def test_gauge_covariance_of_hop():
    dims = (4, 4, 2, 6)
    u = synthetic.gauge_field(dims, eps=0.45, seed=11)
    g = synthetic.random_gauge_transform(dims, seed=12)
    psi = synthetic.random_spinor(dims, seed=13)
    ug = _gauge_transform_links(u, g)
    gpsi = psi @ g.swapaxes(-1, -2)  # (g psi)[s, a] = sum_b g[a, b] psi[s, b]
    lhs = wilson.hop(ug, gpsi, TBC)
    rhs = wilson.hop(u, psi, TBC) @ g.swapaxes(-1, -2)
    assert np.abs(lhs - rhs).max() < 1e-12


def _point_block(fn, dims, site_xyzt):
    """12x12 block (fn)(x, x) at site x from fn applied to the 12 unit sources there."""
    lx, ly, lz, lt = dims
    x, y, z, t = site_xyzt
    src = np.zeros((12,) + lattice.spinor_shape(dims), dtype=np.complex128)
    for s in range(12):
        src[s, t, z, y, x, s // 3, s % 3] = 1.0
    out = fn(src)
    return out[:, t, z, y, x].reshape(12, 12).T  # [row (beta b), col (alpha a)]


def _path_sum_d4(u, dims, site):
    """D^4(x, x) by brute-force enumeration of all closed 4-step paths.

    Step d = +mu carries (1 - gamma_mu) x U_mu(y); d = -mu carries
    (1 + gamma_mu) x U_mu(y - mu)^dagger; crossing the time boundary gives -1.
    """
    lx, ly, lz, lt = dims
    ext = (lx, ly, lz, lt)
    g = lattice.gammas()
    one = np.eye(4)
    steps = [(mu, s) for mu in range(4) for s in (+1, -1)]
    total = np.zeros((12, 12), dtype=np.complex128)
    for path in itertools.product(steps, repeat=4):
        disp = np.zeros(4, dtype=int)
        for mu, s in path:
            disp[mu] += s
        if np.any(disp != 0):
            continue
        spin = np.eye(4, dtype=np.complex128)
        col = np.eye(3, dtype=np.complex128)
        sign = 1.0
        pos = list(site)
        for mu, s in path:
            if s > 0:
                spin = spin @ (one - g[mu])
                link = u[pos[3], pos[2], pos[1], pos[0], mu]
                if mu == 3 and pos[3] == lt - 1:
                    sign *= TBC
                pos[mu] = (pos[mu] + 1) % ext[mu]
                col = col @ link
            else:
                spin = spin @ (one + g[mu])
                if mu == 3 and pos[3] == 0:
                    sign *= TBC
                pos[mu] = (pos[mu] - 1) % ext[mu]
                link = u[pos[3], pos[2], pos[1], pos[0], mu].conj().T
                col = col @ link
        total += sign * np.kron(spin, col)
    return total


def test_hopping_expansion_low_orders_and_plaquette_term():
    dims = (6, 6, 6, 6)
    u = synthetic.gauge_field(dims, eps=0.45, seed=21)
    site = (1, 4, 2, 5)  # (x, y, z, t): t = 5 = T-1 exercises the boundary sign

    def d_n(n):
        def f(src):
            v = src
            for _ in range(n):
                v = wilson.hop(u, v, TBC)
            return v
        return f

    for n in (1, 2, 3):
        assert np.abs(_point_block(d_n(n), dims, site)).max() < 1e-13
    d4 = _point_block(d_n(4), dims, site)
    ref = _path_sum_d4(u, dims, site)
    assert np.abs(d4 - ref).max() < 1e-12
    # Gamma = 1: every oriented plaquette contributes spin trace -8 times the colour
    # trace of its links, so Tr D^4(x,x) = -8 * sum over the 48 oriented plaquettes.
    g = lattice.gammas()
    one = np.eye(4)
    for mu in range(4):
        for nu in range(4):
            if mu != nu:
                for smu in (1, -1):
                    for snu in (1, -1):
                        p = [one - smu * g[mu], one - snu * g[nu], one + smu * g[mu], one + snu * g[nu]]
                        assert abs(np.trace(p[0] @ p[1] @ p[2] @ p[3]) + 8) < 1e-13


def test_free_field_kappa4_coefficient():
    """Free field: Tr M^{-1}(x,x) = 12 - 1152 kappa^4 + O(kappa^6) (48 plaquettes x 3 x -8)."""
    dims = (6, 6, 6, 6)
    k1, k2 = 0.01, 0.005
    c1 = (_free_trace_closed_form(dims, k1) - 12.0) / k1 ** 4
    c2 = (_free_trace_closed_form(dims, k2) - 12.0) / k2 ** 4
    # remove the kappa^2 * C6 term by Richardson extrapolation
    c0 = (c2 * k1 ** 2 - c1 * k2 ** 2) / (k1 ** 2 - k2 ** 2)
    assert abs(c0 + 1152) < 0.5


@pytest.mark.parametrize("eps,target", [(0.45, 0.57), (0.30, 0.79)])
def test_synthetic_plaquette(eps, target):
    u = synthetic.gauge_field((8, 8, 8, 8), eps=eps, seed=1)
    assert abs(wilson.plaquette(u) - target) < 0.02
    # links are SU(3)
    uu = u.reshape(-1, 3, 3)[:100]
    assert np.allclose(uu @ uu.conj().swapaxes(-1, -2), np.eye(3), atol=1e-14)
    assert np.allclose(np.linalg.det(uu), 1.0, atol=1e-14)
