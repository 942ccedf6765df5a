"""Loop contraction, exact loops and the truncated solver method vs the oracle (GPU).

Loops: relative error ||L_gpu - L_oracle|| / ||L_oracle|| per Gamma over the
timeslices, with Gammas whose loop is below 1e-6 of ||L_1|| judged against that
floor; the target is 1e-9 at a final residual of 1e-12.
"""

import numpy as np
import pytest

import synthetic
from oracle import loops, noise, smear, wilson

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def loop_error(got, ref):
    """max over Gamma of ||got_G - ref_G|| / max(||ref_G||, 1e-6 ||ref_1||)."""
    floor = 1e-6 * np.linalg.norm(ref[0])
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.maximum(np.linalg.norm(ref, axis=-1), floor)
    return float((num / den).max())


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 2, 4, 8)])
def test_trace_loops_local_and_smeared(lib, dims):
    U = synthetic.gauge_field(dims, eps=0.45, seed=2)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(0.12)
    eta = synthetic.random_spinor(dims, seed=1, n=5)
    phi = synthetic.random_spinor(dims, seed=2, n=5)
    got = c.trace_loops(to_gpu(eta), to_gpu(phi), lib.SINK_LOCAL | lib.SINK_SMEARED, smear=(4.0, 6))
    ref_l = loops.stochastic_loops(eta, phi)
    ref_s = loops.smeared_loops(U, eta, phi, 4.0, 6)
    assert np.abs(got[:, 0] - ref_l).max() < 1e-12 * np.abs(ref_l).max()
    assert np.abs(got[:, 1] - ref_s).max() < 1e-12 * np.abs(ref_s).max()
    summed = c.trace_loops(to_gpu(eta), to_gpu(phi), lib.SINK_LOCAL, sum_rhs=True)
    assert np.abs(summed[0, 0] - ref_l.sum(0)).max() < 1e-12 * np.abs(ref_l).max()
    # the library's timeslice sums, per pair and over all pairs
    tot = c.trace_loops(to_gpu(eta), to_gpu(phi), lib.SINK_LOCAL | lib.SINK_SMEARED, smear=(4.0, 6), sum_t=True)
    assert tot.shape == (5, 2, 16, 1)
    assert np.abs(tot[:, 0, :, 0] - ref_l.sum(-1)).max() < 1e-12 * np.abs(ref_l.sum(-1)).max()
    assert np.abs(tot[:, 1, :, 0] - ref_s.sum(-1)).max() < 1e-12 * np.abs(ref_s.sum(-1)).max()
    both = c.trace_loops(to_gpu(eta), to_gpu(phi), lib.SINK_LOCAL, sum_rhs=True, sum_t=True)
    assert np.abs(both[0, 0, :, 0] - ref_l.sum((0, -1))).max() < 1e-12 * np.abs(ref_l.sum((0, -1))).max()
    part = c.trace_loops(to_gpu(eta), to_gpu(phi), lib.SINK_LOCAL, t_range=(1, 3))
    assert np.all(part[:, 0, :, 0] == 0) and np.abs(part[:, 0, :, 1:3] - ref_l[:, :, 1:3]).max() < 1e-12 * np.abs(ref_l).max()
    c.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_loops_4x4x4x4(lib, prec):
    """All 12V point sources on 4^4, kappa = 0.10, eps = 0.3: Tr[Gamma M^-1(x,x)] per timeslice."""
    w = synthetic.WORKLOADS["exact_4x4x4x4"]
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    c = lib.Context(w["dims"])
    c.load_gauge(U)
    c.set_kappa(w["kappa"])
    got, st = c.exact_loops(0, 12 * 256, lib.Params(tol=w["tol"], precision=prec, batch=64), lib.SINK_LOCAL)
    ref = loops.exact_loops_dense(U, w["kappa"], -1.0)
    assert st["status"] == 0 and st["true_residual"] <= w["tol"]
    assert loop_error(got[0], ref) < 1e-9
    c.close()


def test_exact_smeared_loops_small(lib):
    dims, kappa = (2, 2, 2, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.5, seed=4)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    got, st = c.exact_loops(0, 12 * 32, lib.Params(tol=1e-12, precision=0, batch=32),
                            lib.SINK_LOCAL | lib.SINK_SMEARED, smear=(2.0, 3))
    assert loop_error(got[0], loops.exact_loops_dense(U, kappa, -1.0)) < 1e-9
    assert loop_error(got[1], loops.exact_smeared_loops_dense(U, kappa, 2.0, 3, -1.0)) < 1e-9
    c.close()


def test_stochastic_loops_end_to_end(lib):
    """Sources -> F32 mixed solve to 1e-12 -> local + smeared loops vs the oracle chain."""
    dims, kappa = (4, 4, 4, 8), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=6)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    dil = noise.SPIN | noise.COLOUR | noise.TIME
    eta = c.make_sources(seed=3, noise_first=2, n_noise=1, dilution=dil, t0=-1)
    phi, st = c.solve(eta, lib.Params(tol=1e-12, precision=1, batch=16))
    got = c.trace_loops(eta, phi, lib.SINK_LOCAL | lib.SINK_SMEARED, smear=(4.0, 50))
    eta_r = noise.make_sources(dims, 3, 2, 1, dil, t0=-1)
    phi_r = np.stack([wilson.solve(U, e, kappa, -1.0, tol=1e-13)[0] for e in eta_r])
    ref_l = loops.stochastic_loops(eta_r, phi_r).sum(0)
    ref_s = loops.smeared_loops(U, eta_r, phi_r, 4.0, 50).sum(0)
    assert loop_error(got[:, 0].sum(0), ref_l) < 1e-9
    assert loop_error(got[:, 1].sum(0), ref_s) < 1e-9
    c.close()


def test_tsm_deterministic_and_combination(lib):
    dims, kappa = (4, 4, 4, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=7)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    lp = lib.Params(precision=2, fixed_iters=6, batch=8)
    hp = lib.Params(tol=1e-11, precision=1, batch=8)
    dil = noise.SPIN | noise.TIME
    a = c.tsm_estimate(11, 6, 3, dil, -1, lp, hp, lib.SINK_LOCAL, per_noise=True)
    b = c.tsm_estimate(11, 6, 3, dil, -1, lp, hp, lib.SINK_LOCAL, per_noise=True)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[0], b[0])
    pn = a[2][:, 0]
    T = dims[3]
    cover = lambda first, n: np.array([[(first + i) % T == t for t in range(T)] for i in range(n)])  # noqa: E731
    mean, var = loops.tsm_estimate(pn[:6], pn[6:9], pn[9:12], lp_cover=cover(0, 6), hp_cover=cover(6, 3))
    assert np.allclose(a[0][0], mean, rtol=1e-12, atol=1e-12)
    assert np.allclose(a[1][0].real + a[1][0].imag, var, rtol=1e-10, atol=1e-12)
    # the HP loops are the exact stochastic loops of those noise vectors
    eta = noise.make_sources(dims, 11, 6, 3, dil, t0=-1)
    phi = np.stack([wilson.solve(U, e, kappa, -1.0, tol=1e-13)[0] for e in eta])
    ref = loops.stochastic_loops(eta, phi).reshape(3, 4, 16, T).sum(1)
    assert loop_error(pn[6:9].reshape(-1, T), ref.reshape(-1, T)) < 1e-8
    c.close()


def test_trace_loops_per_rhs_timeslice_and_groups(lib):
    """Time-diluted sources contracted on their own timeslice, summed per noise vector."""
    dims, kappa = (4, 4, 2, 8), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=9)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    dil = noise.SPIN | noise.COLOUR | noise.TIME
    eta = c.make_sources(seed=5, noise_first=3, n_noise=6, dilution=dil, t0=-1)  # 72 sources, t0 = n mod 8
    phi = torch.from_numpy(synthetic.random_spinor(dims, seed=4, n=72)).cuda()
    t_of = [(3 + j // 12) % 8 for j in range(72)]
    got = c.trace_loops(eta, phi, lib.SINK_LOCAL | lib.SINK_SMEARED, smear=(3.0, 7), t_of_rhs=t_of, group=12)
    assert got.shape == (6, 2, 16, 8)
    e, f = eta.cpu().numpy(), phi.cpu().numpy()
    ref_l = loops.stochastic_loops(e, f)
    ref_s = loops.smeared_loops(U, e, f, 3.0, 7)
    for g in range(6):
        t0 = (3 + g) % 8
        want_l = np.zeros((16, 8), complex)
        want_s = np.zeros((16, 8), complex)
        want_l[:, t0] = ref_l[12 * g:12 * g + 12, :, t0].sum(0)
        want_s[:, t0] = ref_s[12 * g:12 * g + 12, :, t0].sum(0)
        assert np.abs(got[g, 0] - want_l).max() < 1e-12 * np.abs(ref_l).max()
        assert np.abs(got[g, 1] - want_s).max() < 1e-12 * np.abs(ref_s).max()
    # groups of 36 (a batch holds one group) and of 72 (spans batches) agree with the sums
    g36 = c.trace_loops(eta, phi, lib.SINK_LOCAL, t_of_rhs=t_of, group=36)
    assert np.allclose(g36[:, 0], got[:, 0].reshape(2, 3, 16, 8).sum(1), rtol=1e-13, atol=1e-13)
    one = c.trace_loops(eta, phi, lib.SINK_LOCAL, t_of_rhs=t_of, group=72)
    assert np.allclose(one[0, 0], got[:, 0].sum(0), rtol=1e-13, atol=1e-13)
    c.close()


def test_tsm_time_diluted_smeared(lib):
    """TSM with time dilution by translation and a smeared sink: HP loops equal the oracle's."""
    dims, kappa = (4, 4, 4, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=10)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    lp = lib.Params(precision=2, fixed_iters=5, batch=8)
    hp = lib.Params(tol=1e-11, precision=1, batch=8)
    dil = noise.SPIN | noise.TIME
    mean, var, pn = c.tsm_estimate(2, 4, 2, dil, -1, lp, hp, lib.SINK_LOCAL | lib.SINK_SMEARED, smear=(2.0, 4),
                                   per_noise=True)
    eta = noise.make_sources(dims, 2, 4, 2, dil, t0=-1)
    phi = np.stack([wilson.solve(U, e, kappa, -1.0, tol=1e-13)[0] for e in eta])
    ref_s = loops.smeared_loops(U, eta, phi, 2.0, 4).reshape(2, 4, 16, 4).sum(1)
    ref_l = loops.stochastic_loops(eta, phi).reshape(2, 4, 16, 4).sum(1)
    assert loop_error(pn[4:6, 0].reshape(-1, 4), ref_l.reshape(-1, 4)) < 1e-8
    assert loop_error(pn[4:6, 1].reshape(-1, 4), ref_s.reshape(-1, 4)) < 1e-8
    c.close()


def golden_exact_4x4x4x4():
    """The oracle's exact loops of the 4^4 workload (tests/golden, written by make_golden.py)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "exact_loops_4x4x4x4.txt")
    out = np.zeros((16, 4), dtype=np.complex128)
    for g, t, re, im in np.loadtxt(path):
        out[int(g), int(t)] = re + 1j * im
    return out


@pytest.mark.parametrize("dil, n_noise", [(16, 12), (1 | 16, 6), (1 | 2 | 4 | 16, 4)])
def test_dilution_error_matches_oracle(lib, dil, n_noise):
    """The dilution study (Sec. 3, Figs. 3-4) on the 4^4 workload: per-noise loop estimates and the
    per-Gamma mean squared deviation from the exact loops, GPU (FP32 inner, 1e-12) against the
    oracle's estimator on the same noise vectors (bit-identical sources, oracle solves to 1e-13)."""
    w = synthetic.WORKLOADS["exact_4x4x4x4"]
    dims, kappa = w["dims"], w["kappa"]
    U = synthetic.gauge_field(dims, w["eps"], w["seed"])
    exact = golden_exact_4x4x4x4()
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    sig, per = c.dilution_error(9, n_noise, dil, -1, lib.Params(tol=1e-12, precision=1, batch=32), exact,
                                per_noise=True)
    t_of = [n % dims[3] for n in range(n_noise)]
    ref_per = []
    for n in range(n_noise):
        eta = noise.make_sources(dims, 9, n, 1, dil, t0=-1)
        phi = np.stack([wilson.solve(U, e, kappa, -1.0, tol=1e-13)[0] for e in eta])
        ref_per.append(loops.stochastic_loops(eta, phi).sum(0))
    ref_per = np.array(ref_per)
    ref_sig = loops.dilution_sigma2(ref_per, exact, t_of)
    for n in range(n_noise):
        assert loop_error(per[n], ref_per[n]) < 1e-9
    assert np.all(np.abs(sig - ref_sig) <= 1e-8 * ref_sig + 1e-12 * np.abs(exact).max() ** 2), (sig, ref_sig)
    c.close()
