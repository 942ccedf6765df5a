"""Momentum-projected loops, the disconnected correlator and the connected
meson correlator (oracle; test infrastructure).

Sec. 3 builds two-point functions from the loops: the connected function of
Eq. 1 and the disconnected contribution of Eq. 3.  For the eta' (Eq. 4 and
after), the correlator is C_pi - 2D.  The momentum phases sit inside the
operators Gamma_A(p) and Gamma_B(p).  Readings taken here (the printed Eq. 3
is a single trace of two loop propagators and swaps the times of Eq. 1):

* the loop at momentum p = 2 pi n / L (n integer, spatial) is
      L_Gamma(p, t) = sum_{x: x_4 = t} exp(-i p.x) Tr[Gamma S(x, x)];
* the disconnected function is the product of two such traces,
      D^{BA}(p, dt) = -(1 / (L^3 T)) sum_t L_B(p, t + dt) L_A(-p, t),
  with Gamma_B at the later time as in Eq. 1;
* the connected function from one point source at y (Eq. 1 with the sum over
  y replaced by the single source, which is translation-invariant on
  average) is
      C^{BA}(p, dt) = - sum_x exp(-i p.(x - y)) Tr[S(y; x) Gamma_B S(x; y) Gamma_A],
  evaluated with S(y; x) = g5 S(x; y)^dag g5 (gamma5-hermiticity), so it
  needs only the 12 solutions of the point source.  For Gamma_A = Gamma_B =
  g5 this is -sum_x Tr[S^dag S], which is negative in this sign convention.
  The ratio D/C_pi of Eq. 4 does not depend on the common sign.

Pins (tests/test_oracle_correlators.py): p = 0 reduces to the loops of
``loops``.  Exact loops on a translated gauge field pick up the phase
exp(i p_x).  A free field has no loop at p != 0.  The free point-source
propagator built from numpy's FFT of the momentum-space Wilson propagator
gives the same connected correlator as the solver-based one.
"""

from __future__ import annotations

import numpy as np

from .lattice import coordinates, gamma5, spinor_shape, volume
from .wilson import solve


def momentum_phases(dims, momenta) -> np.ndarray:
    """exp(-i p.x) for each momentum n (p_i = 2 pi n_i / L_i) at every site: [P][T][Z][Y][X]."""
    lx, ly, lz, _ = dims
    x, y, z, _ = coordinates(dims)
    out = []
    for n in momenta:
        arg = 2.0 * np.pi * (n[0] * x / lx + n[1] * y / ly + n[2] * z / lz)
        out.append(np.exp(-1j * arg))
    return np.array(out)


def momentum_loops(eta: np.ndarray, phi: np.ndarray, momenta, gammas16: np.ndarray) -> np.ndarray:
    """Per right-hand side n: sum_{x in t} exp(-i p.x) eta_n(x)^dag Gamma phi_n(x), [n][P][16][T]."""
    dims = (eta.shape[-3], eta.shape[-4], eta.shape[-5], eta.shape[-6])
    ph = momentum_phases(dims, momenta)  # [P][T][Z][Y][X]
    # S[n, P, t, beta, alpha] = sum_x phase * sum_a phi[beta, a] conj(eta[alpha, a])
    S = np.einsum("ptzyx,ntzyxba,ntzyxca->nptbc", ph, phi, eta.conj())
    # L_Gamma = sum_{alpha beta} Gamma_{alpha beta} S_{beta alpha}
    return np.einsum("gcb,nptbc->npgt", gammas16, S)


def exact_momentum_loops_dense(U, kappa, momenta, gammas16, t_bc=-1.0) -> np.ndarray:
    """L_Gamma(p, t) from the diagonal blocks of the dense inverse: [P][16][T]."""
    from .wilson import dense_matrix
    lt, lz, ly, lx = U.shape[:4]
    dims = (lx, ly, lz, lt)
    minv = np.linalg.inv(dense_matrix(U, kappa, t_bc, dims))
    blocks = np.array([minv[12 * i:12 * i + 12, 12 * i:12 * i + 12] for i in range(volume(dims))])
    # spin-colour block (beta b, alpha a) -> spin matrix sum_a over colour diagonal
    spin = blocks.reshape(-1, 4, 3, 4, 3).trace(axis1=2, axis2=4)  # [V][beta][alpha]
    spin = spin.reshape(lt, lz, ly, lx, 4, 4)
    ph = momentum_phases(dims, momenta)
    S = np.einsum("ptzyx,tzyxba->ptba", ph, spin)
    return np.einsum("gab,ptba->pgt", gammas16, S)


def disconnected(loops_b: np.ndarray, loops_a_minus_p: np.ndarray, spatial_volume: int) -> np.ndarray:
    """D(dt) = -(1 / (L^3 T)) sum_t L_B(p, t + dt) L_A(-p, t) for loop arrays [..., T]."""
    T = loops_b.shape[-1]
    out = np.zeros(loops_b.shape[:-1] + (T,), dtype=np.complex128)
    for dt in range(T):
        out[..., dt] = -(np.roll(loops_b, -dt, axis=-1) * loops_a_minus_p).sum(-1) / (spatial_volume * T)
    return out


def disconnected_pairs(loops: np.ndarray, cover, minus, spatial_volume: int) -> np.ndarray:
    """D^{BA}(q, dt) from per-noise loops [n][Q][16][T], averaged over ordered pairs
    (n, m), n != m, with n covering t + dt and m covering t:
        D = -(1 / (L^3 T)) sum_t mean_{pairs} L^n_B(q, t + dt) L^m_A(-q, t).
    cover: bool [n][T] (None: all); minus[q]: index of -q.  Returns [Q][16 A][16 B][T]."""
    n, Q, _, T = loops.shape
    cover = np.ones((n, T), dtype=bool) if cover is None else np.asarray(cover, dtype=bool)
    out = np.zeros((Q, 16, 16, T), dtype=np.complex128)
    for q in range(Q):
        for dt in range(T):
            acc = np.zeros((16, 16), dtype=np.complex128)  # [A][B]
            for t in range(T):
                t2 = (t + dt) % T
                pairs = [(a, b) for a in range(n) for b in range(n) if a != b and cover[a, t2] and cover[b, t]]
                if not pairs:
                    continue
                s = sum(np.outer(loops[b, minus[q], :, t], loops[a, q, :, t2]) for a, b in pairs)
                acc += s / len(pairs)
            out[q, :, :, dt] = -acc / (spatial_volume * T)
    return out


def point_propagator(U, kappa, src, t_bc=-1.0, tol=1e-13) -> np.ndarray:
    """The 12 solutions M phi = e_{src, alpha, a}: [12 = 3 alpha + a][T][Z][Y][X][4][3]."""
    lt, lz, ly, lx = U.shape[:4]
    dims = (lx, ly, lz, lt)
    out = []
    for j in range(12):
        e = np.zeros(spinor_shape(dims), dtype=np.complex128)
        e[src[3], src[2], src[1], src[0], j // 3, j % 3] = 1.0
        out.append(solve(U, e, kappa, t_bc, tol=tol)[0])
    return np.array(out)


def connected(prop: np.ndarray, src, momenta, gammas16: np.ndarray) -> np.ndarray:
    """C^{BA}(p, t) for all Gamma_A (source) and Gamma_B (sink): [P][16 A][16 B][T].

    prop[j = 3 alpha + a][x][beta][b] = S(x; y)_{beta b, alpha a}.
    C^{BA} = -sum_x exp(-i p.(x - y)) Tr[g5 S(x)^dag g5 Gamma_B S(x) Gamma_A], t measured from y_4.
    """
    nj, lt, lz, ly, lx = prop.shape[:5]
    dims = (lx, ly, lz, lt)
    S = prop.reshape(4, 3, lt, lz, ly, lx, 4, 3)            # [alpha][a][x][beta][b]
    S = np.moveaxis(S, (0, 1), (-2, -1))                     # [x][beta][b][alpha][a]
    S = S.reshape(lt, lz, ly, lx, 12, 12)                    # S[x][(beta b)][(alpha a)]
    g5 = np.kron(gamma5(), np.eye(3))
    ph = momentum_phases(dims, momenta)
    shift = momentum_phases(dims, momenta)[:, src[3], src[2], src[1], src[0]]  # exp(-i p.y)
    ph = ph / shift[:, None, None, None, None]
    out = np.zeros((len(momenta), 16, 16, lt), dtype=np.complex128)
    Sd = g5 @ np.conj(np.swapaxes(S, -1, -2)) @ g5            # g5 S^dag g5 per site
    for A in range(16):
        GA = np.kron(gammas16[A], np.eye(3))
        for B in range(16):
            GB = np.kron(gammas16[B], np.eye(3))
            tr = np.einsum("tzyxij,jk,tzyxkl,li->tzyx", Sd, GB, S, GA)
            out[:, A, B, :] = -np.einsum("ptzyx,tzyx->pt", ph, tr)
    return np.roll(out, -src[3], axis=-1)


def free_point_propagator(dims, kappa, src, t_bc=-1.0) -> np.ndarray:
    """Free-field (U = 1) point propagator from numpy's FFT of the momentum-space
    Wilson propagator [1 - kappa sum_mu ((1 - g_mu) e^{i k_mu} + (1 + g_mu) e^{-i k_mu})]^{-1},
    with k_4 = (2 m + 1) pi / T for antiperiodic time: same layout as point_propagator."""
    from .lattice import gammas
    lx, ly, lz, lt = dims
    g = gammas()
    one = np.eye(4)
    kx = 2 * np.pi * np.arange(lx) / lx
    ky = 2 * np.pi * np.arange(ly) / ly
    kz = 2 * np.pi * np.arange(lz) / lz
    shift_t = 0.5 if t_bc < 0 else 0.0
    kt = 2 * np.pi * (np.arange(lt) + shift_t) / lt
    Sk = np.zeros((lt, lz, ly, lx, 4, 4), dtype=np.complex128)
    for it, k4 in enumerate(kt):
        for iz, k3 in enumerate(kz):
            for iy, k2 in enumerate(ky):
                for ix, k1 in enumerate(kx):
                    D = np.zeros((4, 4), dtype=np.complex128)
                    for mu, k in enumerate((k1, k2, k3, k4)):
                        D += (one - g[mu]) * np.exp(1j * k) + (one + g[mu]) * np.exp(-1j * k)
                    Sk[it, iz, iy, ix] = np.linalg.inv(one - kappa * D)
    # S(x; 0) = (1/V) sum_k exp(i k.x) S(k): inverse FFT over the periodic momenta,
    # times exp(i pi t / T) for the antiperiodic shift in time
    Sx = np.fft.ifftn(Sk, axes=(0, 1, 2, 3))
    t = np.arange(lt)
    Sx = Sx * np.exp(1j * np.pi * shift_t * 2 * t / lt)[:, None, None, None, None, None]
    # translate the source from the origin to src
    Sx = np.roll(Sx, shift=(src[3], src[2], src[1], src[0]), axis=(0, 1, 2, 3))
    if t_bc < 0 and src[3] != 0:
        # a source at t_y: sites that wrapped across the time boundary change sign
        wrap = np.arange(lt) < src[3]
        Sx[wrap] *= -1.0
    # [x][beta][alpha] (colour identity) -> [12 = 3 alpha + a][x][beta][b]
    out = np.zeros((12, lt, lz, ly, lx, 4, 3), dtype=np.complex128)
    for al in range(4):
        for a in range(3):
            out[3 * al + a, ..., :, a] = Sx[..., :, al]
    return out
