"""Disconnected loops: contraction, exact loops, TSM and gradients (oracle; test infrastructure).

Sec. 3, Eq. 2 of the paper: the disconnected contribution is built from the
loop Tr[S_F(x, x) Gamma] with S_F = M^{-1}; the study inspects its
zero-momentum projection, i.e. the sum over the sites of a timeslice,

    L_Gamma(t) = sum_{x : x_4 = t} Tr_{spin, colour}[ Gamma M^{-1}(x, x) ].

* Exact loops (Sec. 1 and 2, the all-to-all diagonal): M^{-1}(x, x) is the
  12 x 12 diagonal block of the inverse; here from a dense LAPACK inverse
  (tiny lattices) or from 12 point-source solves per site.
* Stochastic loops (Sec. 2): with sources eta and solutions phi = M^{-1} eta,
  the estimate is sum_{x in t} eta(x)^dagger Gamma phi(x), unbiased because
  E[xi xi^dagger] = 1 for complex Z2 noise.  It is assembled from the 4 x 4
  spin matrix S(t)_{beta alpha} = sum_{x in t, a} phi_{beta a}(x) eta*_{alpha a}(x)
  as L_Gamma(t) = sum_{alpha beta} Gamma_{alpha beta} S(t)_{beta alpha}.
* Smeared sinks (Sec. 2): the same with K eta and K phi (K the Gaussian
  smearing operator), an estimate of sum_{x in t} Tr[Gamma (K M^{-1} K)(x, x)].
* Truncated solver method (Sec. 2, after Bali et al.): a large low-precision
  ensemble plus a high-precision bias correction on a separate small ensemble,
  T = mean_LP[eta^dag Gamma f_LP(eta)] + mean_HP[eta^dag Gamma (f_HP - f_LP)(eta)].
"""

from __future__ import annotations

import numpy as np

from .lattice import gamma_basis, spinor_shape, volume
from . import wilson
from .smear import smear


def spin_matrix(eta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """S(t)_{beta alpha} = sum_{x in t} sum_a phi_{beta a}(x) conj(eta_{alpha a}(x)).

    eta, phi: [..., T, Lz, Ly, Lx, 4, 3].  Returns [..., T, 4, 4].
    """
    return np.einsum("...tzyxba,...tzyxca->...tbc", phi, eta.conj())


def trace_gamma(S: np.ndarray) -> np.ndarray:
    """L_Gamma(t) = sum_{alpha beta} Gamma_{alpha beta} S(t)_{beta alpha}.  [..., T, 4, 4] -> [..., 16, T]."""
    return np.einsum("gab,...tba->...gt", gamma_basis(), S)


def stochastic_loops(eta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """sum_{x in t} eta(x)^dagger Gamma phi(x) for all 16 Gamma: [..., 16, T]."""
    return trace_gamma(spin_matrix(eta, phi))


def smeared_loops(U, eta, phi, alpha: float, n_iter: int) -> np.ndarray:
    """sum_{x in t} (K eta)(x)^dagger Gamma (K phi)(x): [..., 16, T]."""
    return stochastic_loops(smear(U, eta, alpha, n_iter), smear(U, phi, alpha, n_iter))


def _diag_blocks_trace(minv: np.ndarray, dims) -> np.ndarray:
    """sum_{x in t} Tr[Gamma A(x, x)] for a dense 12V x 12V matrix A."""
    lx, ly, lz, lt = dims
    v = volume(dims)
    blocks = minv.reshape(v, 4, 3, v, 4, 3)
    idx = np.arange(v)
    diag = blocks[idx, :, :, idx, :, :]  # [V, 4(beta), 3(b), 4(alpha), 3(a)]
    spin = np.einsum("vbaca->vbc", diag)  # colour trace -> [V, beta, alpha]
    spin = spin.reshape(lt, v // lt, 4, 4).sum(axis=1)
    return np.einsum("gab,tba->gt", gamma_basis(), spin)


def exact_loops_dense(U, kappa: float, t_bc: float = -1.0) -> np.ndarray:
    """Exact L_Gamma(t) from the dense inverse of M (tiny lattices only): [16, T]."""
    lt, lz, ly, lx = U.shape[:4]
    dims = (lx, ly, lz, lt)
    m = wilson.dense_matrix(U, kappa, t_bc, dims)
    return _diag_blocks_trace(np.linalg.inv(m), dims)


def smear_matrix(U, alpha: float, n_iter: int) -> np.ndarray:
    """The smearing operator K as a dense 12V x 12V matrix (tiny lattices only)."""
    lt, lz, ly, lx = U.shape[:4]
    dims = (lx, ly, lz, lt)
    n = 12 * volume(dims)
    unit = np.eye(n, dtype=np.complex128).reshape((n,) + spinor_shape(dims))
    return smear(U, unit, alpha, n_iter).reshape(n, n).T.copy()


def exact_smeared_loops_dense(U, kappa, alpha, n_iter, t_bc=-1.0) -> np.ndarray:
    """Exact sum_{x in t} Tr[Gamma (K M^{-1} K)(x, x)] from dense matrices: [16, T]."""
    lt, lz, ly, lx = U.shape[:4]
    dims = (lx, ly, lz, lt)
    m = wilson.dense_matrix(U, kappa, t_bc, dims)
    k = smear_matrix(U, alpha, n_iter)
    return _diag_blocks_trace(k @ np.linalg.solve(m, k), dims)


def point_diagonal_loops(dims, sources_index: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Accumulate sum_{y in t} Tr[Gamma M^{-1}(y, y)] from point-source solutions.

    sources_index[j] = 12*y + 3*alpha + a is the point source solved into phi[j];
    the column phi_j read at its own site y gives M^{-1}(y, y)_{(beta b), (alpha a)}.
    Returns the partial sum over the given sources, [16, T].
    """
    lx, ly, lz, lt = dims
    v = volume(dims)
    spin = np.zeros((lt, 4, 4), dtype=np.complex128)
    flat = phi.reshape(len(sources_index), v, 4, 3)
    for j, s in enumerate(sources_index):
        y, rem = divmod(int(s), 12)
        alpha, a = divmod(rem, 3)
        t = y // (v // lt)
        spin[t, :, alpha] += flat[j, y, :, a]
    return np.einsum("gab,tba->gt", gamma_basis(), spin)


def tsm_estimate(lp: np.ndarray, hp: np.ndarray, lp_on_hp: np.ndarray,
                 lp_cover: np.ndarray | None = None, hp_cover: np.ndarray | None = None):
    """Truncated-solver-method estimate and its variance (Sec. 2, after Bali et al.).

    lp:       [N_LP, 16, T] loops of the low-precision solves on the LP ensemble;
    hp:       [N_HP, 16, T] loops of the high-precision solves on the HP ensemble;
    lp_on_hp: [N_HP, 16, T] loops of the low-precision solves on the HP ensemble.
    *_cover:  optional [N, T] booleans, the timeslices each noise vector covers
              (time dilution); uncovered entries are left out of the averages.

    Returns (mean [16, T], variance of the mean [16, T]):
        mean = <lp> + <hp - lp_on_hp>,  var = s^2(lp)/n_lp + s^2(hp - lp_on_hp)/n_hp
    with per-timeslice sample counts and unbiased sample variances s^2.

    The combination is exact; the low-precision map f_LP that produced lp and
    lp_on_hp is whatever the caller used, and only has to be the same map in both.
    """
    def mean_var(a, cover):
        n_vec = a.shape[0]
        w = np.ones((n_vec, a.shape[-1])) if cover is None else cover.astype(np.float64)
        cnt = w.sum(axis=0)  # [T]
        m = (a * w[:, None, :]).sum(axis=0) / np.maximum(cnt, 1)
        d = (a - m[None]) * w[:, None, :]
        s2 = (np.abs(d) ** 2).sum(axis=0) / np.maximum(cnt - 1, 1)
        return m, s2 / np.maximum(cnt, 1)

    m_lp, v_lp = mean_var(lp, lp_cover)
    m_d, v_d = mean_var(hp - lp_on_hp, hp_cover)
    return m_lp + m_d, v_lp + v_d


def dilution_sigma2(per_noise: np.ndarray, exact: np.ndarray, t_of=None) -> np.ndarray:
    """Stochastic error of one noise vector's loop estimate (the dilution study of Sec. 3, Figs. 3-4).

    per_noise: [n, 16, T] loop estimates, each summed over the dilution classes of one noise
    vector; exact: [16, T] exact loops; t_of: [n] source timeslice of each time-diluted vector
    (None: every timeslice of every vector counts).  Returns, per Gamma, the mean of
    |L_n(t) - exact(t)|^2 over the vectors (and timeslices) that estimate it.  With K classes per
    vector, an estimate costing N_inv inversions has the error sqrt(sigma2 K / N_inv).
    """
    dev = np.abs(per_noise - exact[None]) ** 2  # [n, 16, T]
    if t_of is None:
        return dev.mean(axis=(0, 2))
    return np.array([dev[i, :, t] for i, t in enumerate(t_of)]).mean(axis=0)


def loop_gradients(U, kappa, eta, gamma_index: int, g: np.ndarray, t_bc=-1.0, tol=1e-13):
    """Gradients of a real loss through L(t) = sum_{x in t} eta^dag Gamma M^{-1} eta.

    g[t] is the incoming gradient dloss/dconj(L(t)) (PyTorch's convention for
    complex outputs).  With phi = M^{-1} eta and, for each t,
    chi_t = M^{-dagger} Gamma^dagger P_t eta (P_t: restriction to timeslice t):

        grad_eta   = sum_t [ g_t chi_t + conj(g_t) P_t Gamma phi ]
        grad_kappa = Re sum_t g_t conj(chi_t^dagger D phi)

    since dL/deta* = P_t Gamma phi, dL/deta = conj(chi_t), and
    dM^{-1}/dkappa = M^{-1} D M^{-1} (M = 1 - kappa D).  The sum over t is taken
    inside one adjoint solve: sum_t g_t chi_t = M^{-dagger} Gamma^dagger (g * eta).
    Returns (grad_eta, grad_kappa).
    """
    gam = gamma_basis()[gamma_index]
    lt = eta.shape[0]
    phi, _ = wilson.solve(U, eta, kappa, t_bc, tol=tol)
    g_eta = eta * g.reshape(lt, 1, 1, 1, 1, 1)
    src = np.einsum("sr,...ra->...sa", gam.conj().T, g_eta)
    chi_g, _ = wilson.solve_adjoint(U, src, kappa, t_bc, tol=tol)
    gphi = np.einsum("sr,...ra->...sa", gam, phi) * np.conj(g).reshape(lt, 1, 1, 1, 1, 1)
    grad_eta = chi_g + gphi
    dphi = wilson.hop(U, phi, t_bc)
    # sum_t g_t conj(chi_t^dag D phi) = conj( (sum_t conj(g_t) chi_t)^dag D phi ) ... written per t:
    grad_kappa = 0.0
    for t in range(lt):
        p_eta = np.zeros_like(eta)
        p_eta[t] = eta[t]
        chi_t, _ = wilson.solve_adjoint(U, np.einsum("sr,...ra->...sa", gam.conj().T, p_eta), kappa, t_bc, tol=tol)
        dl_dk = np.vdot(chi_t.ravel(), dphi.ravel())
        grad_kappa += (g[t] * np.conj(dl_dk)).real
    return grad_eta, float(grad_kappa)
