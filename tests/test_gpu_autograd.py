"""LoopTrace autograd (adjoint solve) vs the oracle gradient and finite differences (GPU)."""

import numpy as np
import pytest

import synthetic
from oracle import loops, noise

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def setup(lib, dims, kappa, seed=6):
    U = synthetic.gauge_field(dims, eps=0.45, seed=seed)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    return c, U


def test_gradients_match_oracle(lib):
    from paper_1012_5168_gb300.autograd import loop_trace
    dims, kappa, gidx = (4, 4, 2, 4), 0.12, 5
    c, U = setup(lib, dims, kappa)
    params = lib.Params(tol=1e-13, precision=0, batch=2)
    etas = np.stack([noise.z2_noise(dims, 3, n) for n in range(2)])
    eta = torch.from_numpy(etas).cuda().requires_grad_(True)
    k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    L = loop_trace(eta, k, c, params)
    rng = np.random.default_rng(0)
    cw = torch.from_numpy(rng.standard_normal((2, dims[3])) + 1j * rng.standard_normal((2, dims[3]))).cuda()
    loss = (cw.conj() * L[:, gidx]).real.sum()
    loss.backward()
    ge_tot, gk_tot = 0.0, 0.0
    for j in range(2):
        g = np.zeros(dims[3], dtype=np.complex128)
        # for loss = Re(conj(c) L) PyTorch passes grad_output g = c
        g[:] = cw[j].cpu().numpy()
        ge, gk = loops.loop_gradients(U, kappa, etas[j], gidx, g, -1.0)
        assert np.abs(eta.grad[j].cpu().numpy() - ge).max() < 1e-9 * np.abs(ge).max()
        gk_tot += gk
    assert abs(k.grad.item() - gk_tot) < 1e-8 * abs(gk_tot)
    c.close()


def test_dkappa_central_difference(lib):
    from paper_1012_5168_gb300.autograd import loop_trace
    dims, kappa = (8, 8, 8, 16), 0.14
    c, U = setup(lib, dims, kappa, seed=1)
    params = lib.Params(tol=1e-12, precision=1, batch=16)
    eta = c.make_sources(seed=2, noise_first=0, n_noise=4, dilution=0)
    k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    L = loop_trace(eta, k, c, params)
    loss = L[:, 5].real.sum()  # Tr[g5 M^-1] estimate
    loss.backward()
    dk = 1e-5
    lp = loop_trace(eta, torch.tensor(kappa + dk, dtype=torch.float64), c, params)[:, 5].real.sum()
    lm = loop_trace(eta, torch.tensor(kappa - dk, dtype=torch.float64), c, params)[:, 5].real.sum()
    fd = (lp - lm).item() / (2 * dk)
    assert abs(k.grad.item() - fd) < 1e-5 * abs(fd) + 1e-7
    c.close()


def test_gradcheck_tiny(lib):
    from paper_1012_5168_gb300.autograd import loop_trace
    dims, kappa = (2, 2, 2, 2), 0.1
    c, U = setup(lib, dims, kappa, seed=2)
    params = lib.Params(tol=1e-14, precision=0, batch=1, max_iter=2000)
    eta = torch.from_numpy(synthetic.random_spinor(dims, 1, n=1)).cuda().requires_grad_(True)
    k = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    f = lambda e, kk: loop_trace(e, kk, c, params)  # noqa: E731
    assert torch.autograd.gradcheck(f, (eta, k), eps=1e-6, atol=1e-6, rtol=1e-5, fast_mode=True)
    c.close()
