"""Clover-improved Wilson operator on the device vs the oracle (GPU).

The clover term is an extension beyond the paper's plain Wilson inversions
(Sec. 2); the oracle states its convention and pins it.  Here the library's
A (built on the device from the FP64 links), M = A - kappa D, the even-odd
clover solve in every inner precision, its adjoint and the exact loops that
run through it are compared with the oracle on the same seeded links.
"""

import numpy as np
import pytest

import synthetic
from oracle import clover, loops

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_rows(a, b):
    n = len(a)
    return np.linalg.norm((a - b).reshape(n, -1), axis=1) / np.linalg.norm(b.reshape(n, -1), axis=1)


def test_apply_m_matches_oracle(lib):
    dims, kappa, csw = (4, 4, 6, 8), 0.12, 1.6
    U = synthetic.gauge_field(dims, eps=0.45, seed=41)
    x = synthetic.random_spinor(dims, seed=42, n=3)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    c.set_clover(csw)
    got = c.apply_m(to_gpu(x)).cpu().numpy()
    ref = np.stack([clover.apply_m(U, xx, kappa, csw) for xx in x])
    assert rel_rows(got, ref).max() < 1e-13
    # a new kappa rebuilds A (kappa c_sw enters it)
    c.set_kappa(0.135)
    got = c.apply_m(to_gpu(x)).cpu().numpy()
    ref = np.stack([clover.apply_m(U, xx, 0.135, csw) for xx in x])
    assert rel_rows(got, ref).max() < 1e-13
    # new links rebuild it too
    U2 = synthetic.gauge_field(dims, eps=0.3, seed=43)
    c.load_gauge(U2)
    got = c.apply_m(to_gpu(x)).cpu().numpy()
    ref = np.stack([clover.apply_m(U2, xx, 0.135, csw) for xx in x])
    assert rel_rows(got, ref).max() < 1e-13
    # c_sw = 0 is the Wilson operator again, bit for bit
    c.set_clover(0.0)
    wil = c.apply_m(to_gpu(x)).cpu().numpy()
    c2 = lib.Context(dims)
    c2.load_gauge(U2)
    c2.set_kappa(0.135)
    assert np.array_equal(wil, c2.apply_m(to_gpu(x)).cpu().numpy())
    c.close()
    c2.close()


def test_apply_hop_ignores_clover(lib):
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, eps=0.45, seed=44)
    x = synthetic.random_spinor(dims, seed=45, n=2)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(0.12)
    plain = c.apply_hop(to_gpu(x)).cpu().numpy()
    c.set_clover(1.2)
    assert np.array_equal(plain, c.apply_hop(to_gpu(x)).cpu().numpy())
    c.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("graph", [1, 0])
def test_clover_solve(lib, prec, graph):
    dims, kappa, csw = (4, 4, 4, 8), 0.12, 1.5
    U = synthetic.gauge_field(dims, eps=0.45, seed=46)
    b = synthetic.random_spinor(dims, seed=47, n=5)  # batch 4: a ragged second batch
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    c.set_clover(csw)
    tol = 1e-11
    x, st = c.solve(to_gpu(b), lib.Params(tol=tol, precision=prec, batch=4, use_graph=graph, chunk=3))
    x = x.cpu().numpy()
    assert all(s["status"] == 0 for s in st), st
    res = np.linalg.norm(np.stack([bb - clover.apply_m(U, xx, kappa, csw) for bb, xx in zip(b, x)]).reshape(5, -1),
                         axis=1) / np.linalg.norm(b.reshape(5, -1), axis=1)
    assert np.all(res <= tol), res
    assert all(abs(s["true_residual"] - r) < 0.05 * tol + 1e-3 * r for s, r in zip(st, res))
    ref = np.stack([clover.solve(U, bb, kappa, csw, tol=1e-13)[0] for bb in b[:2]])
    assert np.abs(x[:2] - ref).max() / np.abs(ref).max() < 1e-9
    c.close()


def test_clover_adjoint_solve_and_cgnr_refused(lib):
    dims, kappa, csw = (2, 2, 2, 4), 0.12, 1.7
    U = synthetic.gauge_field(dims, eps=0.5, seed=48)
    b = synthetic.random_spinor(dims, seed=49, n=3)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    c.set_clover(csw)
    m = clover.dense_matrix(U, kappa, csw)
    x, st = c.solve_adjoint(to_gpu(b), lib.Params(tol=1e-12, precision=1, batch=4))
    x = x.cpu().numpy()
    assert all(s["status"] == 0 for s in st), st
    for bb, xx in zip(b, x):
        r = bb.reshape(-1) - m.conj().T @ xx.reshape(-1)
        assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(bb)
    with pytest.raises(lib.DlError) as e:
        c.solve(to_gpu(b), lib.Params(tol=1e-10, precision=1, method=lib.METHOD_CGNR))
    assert e.value.status == 1
    c.close()


def test_clover_exact_loops_4x4x4x4(lib):
    """All 12 V point sources on 4^4 with clover: Tr[Gamma M^-1(x, x)] vs the dense inverse."""
    dims, kappa, csw = (4, 4, 4, 4), 0.11, 1.3
    U = synthetic.gauge_field(dims, eps=0.3, seed=50)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    c.set_clover(csw)
    got, st = c.exact_loops(0, 12 * 256, lib.Params(tol=1e-12, precision=1, batch=64), lib.SINK_LOCAL)
    assert st["status"] == 0 and st["true_residual"] <= 1e-12
    ref = loops._diag_blocks_trace(np.linalg.inv(clover.dense_matrix(U, kappa, csw)), dims)
    floor = 1e-6 * np.linalg.norm(ref[0])
    err = np.linalg.norm(got[0] - ref, axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), floor)
    assert err.max() < 1e-9
    c.close()


def test_apply_clover_and_inverse(lib):
    dims, kappa, csw = (4, 4, 4, 4), 0.13, 1.9
    U = synthetic.gauge_field(dims, eps=0.5, seed=51)
    x = synthetic.random_spinor(dims, seed=52, n=2)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    c.set_clover(csw)
    ax = c.apply_clover(to_gpu(x)).cpu().numpy()
    ref = np.stack([clover.apply_clover(U, xx, kappa, csw) for xx in x])
    assert rel_rows(ax, ref).max() < 1e-14
    back = c.apply_clover(to_gpu(ax), inverse=True).cpu().numpy()
    assert rel_rows(back, x).max() < 1e-13
    c.set_clover(0.0)  # A = 1
    assert np.array_equal(c.apply_clover(to_gpu(x)).cpu().numpy(), x)
    c.close()


def test_dm_dkappa(lib):
    """-dM/dkappa x against the oracle's M, which is linear in kappa: (M(k1) - M(k2)) x / (k2 - k1)."""
    dims, kappa, csw = (4, 2, 4, 8), 0.12, 1.4
    U = synthetic.gauge_field(dims, eps=0.45, seed=53)
    x = synthetic.random_spinor(dims, seed=54, n=2)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    for cs in (csw, 0.0):
        c.set_clover(cs)
        got = c.apply_dm_dkappa(to_gpu(x)).cpu().numpy()
        ref = np.stack([(clover.apply_m(U, xx, 0.1, cs) - clover.apply_m(U, xx, 0.2, cs)) / 0.1 for xx in x])
        assert rel_rows(got, ref).max() < 1e-13
    c.close()


def test_clover_gradcheck_tiny(lib):
    from paper_1012_5168_gb300.autograd import loop_trace
    dims, kappa = (2, 2, 2, 2), 0.1
    U = synthetic.gauge_field(dims, eps=0.5, seed=55)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    c.set_clover(1.6)
    params = lib.Params(tol=1e-14, precision=0, batch=1, max_iter=2000)
    eta = torch.from_numpy(synthetic.random_spinor(dims, 3, n=1)).cuda().requires_grad_(True)
    k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    f = lambda e, kk: loop_trace(e, kk, c, params)  # noqa: E731
    assert torch.autograd.gradcheck(f, (eta, k), eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)
    c.close()


def test_clover_argument_errors(lib):
    """Non-finite c_sw is refused; -dM/dkappa with clover needs kappa != 0; A^-1 A is the identity
    only where A exists, and c_sw = 0 leaves -dM/dkappa = D."""
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, eps=0.4, seed=56)
    x = to_gpu(synthetic.random_spinor(dims, seed=57, n=1))
    c = lib.Context(dims)
    c.load_gauge(U)
    for bad in (float("nan"), float("inf")):
        with pytest.raises(lib.DlError) as e:
            c.set_clover(bad)
        assert e.value.status == 1
    c.set_kappa(0.0)
    c.set_clover(1.0)
    with pytest.raises(lib.DlError) as e:
        c.apply_dm_dkappa(x)
    assert e.value.status == 1
    c.set_clover(0.0)
    assert torch.equal(c.apply_dm_dkappa(x), c.apply_hop(x))
    c.close()
