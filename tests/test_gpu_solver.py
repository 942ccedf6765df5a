"""CUDA even-odd BiCGStab (FP64, FP32- and BF16-inner defect correction) vs the oracle (GPU).

A solve is correct when the oracle's own FP64 M reproduces b from the
solution: ||b - M x|| / ||b|| <= tol, evaluated on the CPU.  Solutions are also
compared with the oracle's full-lattice BiCGStab.
"""

import numpy as np
import pytest

import synthetic
from oracle import krylov, wilson

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def residual(U, x, b, kappa):
    r = b - wilson.apply_m(U, x, kappa, -1.0)
    return np.linalg.norm(r.reshape(len(b), -1), axis=1) / np.linalg.norm(b.reshape(len(b), -1), axis=1)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("graph", [1, 0])
def test_solve_small(lib, prec, graph):
    dims, kappa = (4, 4, 4, 8), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=3)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = synthetic.random_spinor(dims, seed=9, n=5)  # 5 right-hand sides, batch 4: a ragged batch
    tol = 1e-11
    x, st = c.solve(to_gpu(b), lib.Params(tol=tol, precision=prec, batch=4, use_graph=graph, chunk=3))
    x = x.cpu().numpy()
    assert all(s["status"] == 0 for s in st), st
    res = residual(U, x, b, kappa)
    assert np.all(res <= tol), res
    assert all(abs(s["true_residual"] - r) < 0.05 * tol + 1e-3 * r for s, r in zip(st, res))
    ref = np.stack([wilson.solve(U, bb, kappa, -1.0, tol=1e-13)[0] for bb in b[:2]])
    assert np.abs(x[:2] - ref).max() / np.abs(ref).max() < 1e-9
    c.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_float_float_defect_correction(lib, prec, monkeypatch):
    """Residual steps in float-float (the mixed-precision default) and in FP64 both reach tol.

    Both solutions are checked against the oracle's FP64 M on the CPU, and the
    residual the library reports must match that CPU residual.
    """
    dims, kappa = (6, 4, 4, 8), 0.13
    U = synthetic.gauge_field(dims, eps=0.45, seed=31)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = synthetic.random_spinor(dims, seed=32, n=6)
    b[5] *= 1e-7  # right-hand sides far from unit norm, some outside the float exponent range
    b[4] *= 1e-35
    b[3] *= 1e-42
    b[2] *= 1e35
    tol = 1e-10
    sols = []
    for flag in ("1", "0"):
        monkeypatch.setenv("DLOOPS_OUTER_DFF", flag)
        x, st = c.solve(to_gpu(b), lib.Params(tol=tol, precision=prec, batch=8))
        x = x.cpu().numpy()
        assert all(s["status"] == 0 for s in st), st
        res = residual(U, x, b, kappa)
        assert np.all(res <= tol), (flag, res)
        assert all(abs(s["true_residual"] - r) < 0.01 * tol + 1e-3 * r for s, r in zip(st, res)), (flag, st, res)
        sols.append(x)
    monkeypatch.delenv("DLOOPS_OUTER_DFF")
    for j in range(len(b)):
        assert np.abs(sols[0][j] - sols[1][j]).max() < 1e-8 * np.abs(sols[1][j]).max()
    c.close()


def test_graph_and_eager_agree_bitwise(lib):
    """The inner iteration is deterministic: graph replay == direct launches, run twice."""
    dims, kappa = (4, 4, 4, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=1)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = to_gpu(synthetic.random_spinor(dims, seed=2, n=4))
    outs = []
    for graph in (1, 0, 1):
        x, _ = c.solve(b, lib.Params(precision=2, fixed_iters=13, batch=4, use_graph=graph, chunk=5))
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    c.close()


def test_adjoint_solve(lib):
    dims, kappa = (4, 4, 2, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=4)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = synthetic.random_spinor(dims, seed=5, n=2)
    x, st = c.solve_adjoint(to_gpu(b), lib.Params(tol=1e-11, precision=1))
    x = x.cpu().numpy()
    r = b - wilson.apply_mdag(U, x, kappa, -1.0)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-11
    c.close()


def test_edge_cases(lib):
    dims, kappa = (4, 4, 4, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=4)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    # zero source -> zero solution, converged
    z = torch.zeros((2, 4, 4, 4, 4, 4, 3), dtype=torch.complex128, device="cuda")
    x, st = c.solve(z)
    assert torch.count_nonzero(x).item() == 0 and all(s["status"] == 0 for s in st)
    # no right-hand sides
    e = torch.zeros((0, 4, 4, 4, 4, 4, 3), dtype=torch.complex128, device="cuda")
    x, st = c.solve(e)
    assert st == []
    # iteration cap -> NOT_CONVERGED reported, no hang
    b = to_gpu(synthetic.random_spinor(dims, seed=1, n=1))
    with pytest.raises(lib.DlError) as err:
        c.solve(b, lib.Params(tol=1e-12, precision=1, max_iter=3))
    assert err.value.status == lib.NOT_CONVERGED
    x, st = c.solve(b, lib.Params(tol=1e-12, precision=1, max_iter=3), allow_fail=True)
    assert st[0]["status"] == lib.NOT_CONVERGED and st[0]["iters"] <= 3
    c.close()


def test_supercritical_kappa_stops_cleanly(lib):
    """kappa = 0.157 on eps = 0.45 links is past the critical point: the solve gives up."""
    w = synthetic.WORKLOADS["supercritical_8x8x8x16"]
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    c = lib.Context(w["dims"])
    c.load_gauge(U)
    c.set_kappa(w["kappa"])
    b = to_gpu(synthetic.random_spinor(w["dims"], seed=1, n=2))
    x, st = c.solve(b, lib.Params(tol=1e-10, precision=1, max_iter=600), allow_fail=True)
    assert all(s["status"] in (lib.NOT_CONVERGED, lib.BREAKDOWN, lib.NAN) for s in st)
    assert all(s["iters"] <= 600 for s in st)
    c.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solve_full_size(lib, prec):
    """The paper's lattice shape (16^3 x 32), batch 16: residual checked by the oracle on samples."""
    w = synthetic.WORKLOADS["wilson_16x16x16x32"]
    dims, kappa = w["dims"], w["kappa"]
    U = synthetic.gauge_field(dims, w["eps"], w["seed"])
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    n = 16 if prec else 2
    eta = c.make_sources(seed=1, noise_first=0, n_noise=n, dilution=0)
    x, st = c.solve(eta, lib.Params(tol=1e-10, precision=prec, batch=16))
    assert all(s["status"] == 0 for s in st), st
    for j in (0, n - 1):
        b = eta[j:j + 1].cpu().numpy()
        res = residual(U, x[j:j + 1].cpu().numpy(), b, kappa)
        assert res[0] <= 1e-10, res
    c.close()


def plain_f32_layout(monkeypatch, prec, kind):
    """FP32 fields of the contexts made now: paired for kinds 7-9, which read that layout only."""
    if prec == 1 and 7 <= kind <= 9:
        monkeypatch.setenv("DLOOPS_F32_PAIRS", "1")


@pytest.mark.parametrize("prec, kind", [(p, k) for p in (1, 2) for k in (0, 1, 2, 3)] + [(1, 7), (1, 8), (1, 9), (1, 10)])
@pytest.mark.parametrize("batch", [1, 4, 16, 64])
def test_hop_kernel_kinds(lib, prec, kind, batch, monkeypatch):
    """Direct, cp.async-prefetching, bulk-copy-staged and blocked-mapping hops, and the paired-layout
    packed-FP32 hops (kinds 7, 8: FP32 of even width), all solve to tolerance."""
    if 7 <= kind <= 9 and batch == 1:
        pytest.skip("the paired layout holds two right-hand sides per group: even widths only")
    if kind == 9 and batch != 64:
        pytest.skip("the warp-staged paired hop serves widths 32 and 64")
    plain_f32_layout(monkeypatch, prec, kind)
    dims, kappa = (4, 4, 4, 8), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=8)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    # batch - 1 right-hand sides: the layout width is `batch` itself, with a ragged last column
    n = batch - 1 if batch > 1 else 2
    b = synthetic.random_spinor(dims, seed=21, n=n)
    R, B, k, _ = c.tune_hop(prec, batch, force_pf=kind)
    assert k == kind
    x, st = c.solve(to_gpu(b), lib.Params(tol=1e-11, precision=prec, batch=batch))
    assert all(s["status"] == 0 for s in st), st
    res = residual(U, x.cpu().numpy(), b, kappa)
    assert np.all(res <= 1e-11), res
    c.close()


@pytest.mark.parametrize("prec, kind", [(1, 4), (2, 4), (2, 5), (1, 6), (1, 7), (1, 8), (1, 9), (1, 11), (2, 11)])
@pytest.mark.parametrize("batch", [32, 64])
def test_warp_staged_hop_solves(lib, prec, kind, batch, monkeypatch):
    """The warp-staged hops (one site per warp, N = 32 R: kind 4 on the CUDA cores, kind 5 on the
    tensor cores for BF16) and the packed-FP32 direct hop (kind 6) at widths 32 and 64, with a ragged
    last batch, solve to tolerance.  8^3 x 24 has more even sites (6144) than a 152-SM GPU runs warps of
    this kernel (at most 2432), so every warp walks several sites and reuses its stages and link rows.
    Kinds 7 and 8 (paired layout, two right-hand sides per thread) and kind 9 (paired and
    warp-staged, 64 / N sites per warp) run at the same widths."""
    plain_f32_layout(monkeypatch, prec, kind)
    dims, kappa = (8, 8, 8, 24), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=9)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = synthetic.random_spinor(dims, seed=22, n=batch + 3)
    k = [0, batch - 1, batch, batch + 2]  # fields checked with the oracle's M
    R, B, got_kind, _ = c.tune_hop(prec, batch, force_pf=kind)
    assert got_kind == kind and R == {6: 1, 7: 2, 8: 2, 9: 2}.get(kind, batch // 32)
    x, st = c.solve(to_gpu(b), lib.Params(tol=1e-11, precision=prec, batch=batch))
    assert all(s["status"] == 0 and s["true_residual"] <= 1e-11 for s in st), st
    res = residual(U, x.cpu().numpy()[k], b[k], kappa)
    assert np.all(res <= 1e-11), res
    c.close()


def test_hop_kernel_kinds_full_size(lib, monkeypatch):
    """The FP32 hop kernels give the same Schur solve on the 16^3 x 32 lattice (32 right-hand sides):
    kinds 0-4 on the plain layout, kinds 0, 7, 8, 9 on the paired one."""
    w = synthetic.WORKLOADS["wilson_16x16x16x32"]
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    sols = []
    for pairs, kinds in (("0", (0, 1, 2, 3, 4, 10, 11)), ("1", (0, 7, 8, 9))):
        monkeypatch.setenv("DLOOPS_F32_PAIRS", pairs)
        c = lib.Context(w["dims"])
        c.load_gauge(U)
        c.set_kappa(w["kappa"])
        eta = c.make_sources(seed=4, noise_first=0, n_noise=32, dilution=0)
        for kind in kinds:
            c.tune_hop(1, 32, force_pf=kind)
            x, st = c.solve(eta, lib.Params(tol=1e-10, precision=1, batch=32))
            assert all(s["status"] == 0 and s["true_residual"] <= 1e-10 for s in st)
            sols.append(x)
        c.close()
    for x in sols[1:]:
        assert (torch.linalg.vector_norm(x - sols[0]) / torch.linalg.vector_norm(sols[0])).item() < 1e-9


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("k", [1, 7, 25])
def test_fixed_iteration_map_matches_oracle(lib, method, k):
    """FP64 storage, k fixed iterations of BiCGStab (0) or CGNR (1) on the Schur system.

    The GPU iterate, reconstructed on the full lattice, equals the oracle's
    restatement of the same k steps (the low-precision map of the truncated
    solver method, here without the rounding of a low-precision type).
    """
    dims, kappa = (4, 4, 4, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=12)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = synthetic.random_spinor(dims, seed=13, n=3)
    x, st = c.solve(to_gpu(b), lib.Params(precision=0, fixed_iters=k, batch=4, method=method))
    x = x.cpu().numpy()
    op = lambda v: krylov.schur_apply(U, v, kappa)  # noqa: E731
    opd = lambda v: krylov.schur_apply_dag(U, v, kappa)  # noqa: E731
    for j in range(3):
        assert st[j]["iters"] == k
        bhat = krylov.schur_rhs(U, b[j], kappa)
        xe = krylov.cgnr(op, opd, bhat, n_iter=k)[0] if method else krylov.bicgstab_fixed(op, bhat, k)[0]
        ref = krylov.schur_reconstruct(U, xe, b[j], kappa)
        assert np.abs(x[j] - ref).max() < 1e-11 * np.abs(ref).max()
    c.close()


def test_bf16_lp_map_error_bound(lib):
    """30 BF16 BiCGStab iterations (the benchmark's low-precision map) stay within a stated
    bound of the same 30 iterations in FP64: BF16 keeps 8 significand bits, so the map is
    parity-unpinned beyond that bound."""
    dims, kappa = (4, 4, 4, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=14)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = synthetic.random_spinor(dims, seed=15, n=2)
    x, _ = c.solve(to_gpu(b), lib.Params(precision=2, fixed_iters=30, batch=2))
    x = x.cpu().numpy()
    op = lambda v: krylov.schur_apply(U, v, kappa)  # noqa: E731
    for j in range(2):
        bhat = krylov.schur_rhs(U, b[j], kappa)
        ref = krylov.schur_reconstruct(U, krylov.bicgstab_fixed(op, bhat, 30)[0], b[j], kappa)
        err = np.linalg.norm(x[j] - ref) / np.linalg.norm(ref)
        print(f"bf16 30-iteration map: relative difference {err:.3e}")
        assert err < 1e-2
    c.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_cgnr_solve_small(lib, prec):
    """CGNR inner solver with FP64 defect correction: ragged batch, graph and eager."""
    dims, kappa = (4, 4, 4, 8), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=16)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = synthetic.random_spinor(dims, seed=17, n=5)
    for graph in (1, 0):
        x, st = c.solve(to_gpu(b), lib.Params(tol=1e-11, precision=prec, batch=4, use_graph=graph, chunk=5,
                                              method=lib.METHOD_CGNR))
        assert all(s["status"] == 0 for s in st), st
        assert np.all(residual(U, x.cpu().numpy(), b, kappa) <= 1e-11)
    c.close()


def test_cgnr_single_precision_lp_full_size(lib):
    """Sec. 2's low-precision solve on 16^3 x 32: single-precision CG to a 1e-6 tolerance."""
    w = synthetic.WORKLOADS["wilson_16x16x16x32"]
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    c = lib.Context(w["dims"])
    c.load_gauge(U)
    c.set_kappa(w["kappa"])
    eta = c.make_sources(seed=2, noise_first=0, n_noise=16, dilution=0)
    x, st = c.solve(eta, lib.Params(tol=1e-6, precision=1, delta=1e-6, batch=16, method=lib.METHOD_CGNR))
    assert all(s["status"] == 0 and s["true_residual"] <= 1e-6 for s in st), st
    b = eta[:1].cpu().numpy()
    assert residual(U, x[:1].cpu().numpy(), b, w["kappa"])[0] <= 1e-6
    x2, _ = c.solve(eta, lib.Params(tol=1e-6, precision=1, delta=1e-6, batch=16, method=lib.METHOD_CGNR))
    assert torch.equal(x, x2)  # a deterministic map, as the truncated solver method needs
    c.close()


def test_nan_source_reports_nan_and_spares_the_batch(lib):
    """A NaN placed on the host in one source: that right-hand side reports DL_NAN, the others converge."""
    dims, kappa = (4, 4, 4, 4), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=18)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = synthetic.random_spinor(dims, seed=19, n=4)
    b[2, 1, 2, 3, 0, 1, 2] = np.nan
    for prec in (0, 1):
        x, st = c.solve(to_gpu(b), lib.Params(tol=1e-11, precision=prec, batch=4), allow_fail=True)
        assert st[2]["status"] == lib.NAN
        good = [0, 1, 3]
        assert all(st[j]["status"] == 0 for j in good), st
        res = residual(U, x.cpu().numpy()[good], b[good], kappa)
        assert np.all(res <= 1e-11), res
    c.close()


def test_dilution_linearity(lib):
    """Sum over the dilution classes of the solutions equals the solution of the undiluted noise vector."""
    dims, kappa = (4, 4, 2, 8), 0.12
    c = lib.Context(dims)
    c.load_gauge(synthetic.gauge_field(dims, eps=0.45, seed=20))
    c.set_kappa(kappa)
    p = lib.Params(tol=1e-12, precision=1, batch=16)
    dil = lib.DIL_SPIN | lib.DIL_COLOUR | lib.DIL_EVENODD
    eta = c.make_sources(seed=9, noise_first=3, n_noise=1, dilution=dil)  # 24 classes of one vector
    xi = c.make_sources(seed=9, noise_first=3, n_noise=1, dilution=0)
    assert torch.equal(eta.sum(0), xi[0])
    phi, _ = c.solve(eta, p)
    phi_xi, _ = c.solve(xi, p)
    diff = (phi.sum(0) - phi_xi[0]).abs().max().item()
    assert diff < 1e-10 * phi_xi.abs().max().item()
    c.close()


def test_solve_larger_lattice(lib):
    """24^3 x 48 (V = 663,552), 32 right-hand sides: residuals checked with the oracle's M on samples."""
    dims, kappa = (24, 24, 24, 48), 0.14
    U = synthetic.gauge_field(dims, eps=0.45, seed=2)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    eta = c.make_sources(seed=5, noise_first=0, n_noise=32, dilution=0)
    x, st = c.solve(eta, lib.Params(tol=1e-10, precision=1, batch=32))
    assert all(s["status"] == 0 and s["true_residual"] <= 1e-10 for s in st), st
    for j in (0, 31):
        b = eta[j:j + 1].cpu().numpy()
        assert residual(U, x[j:j + 1].cpu().numpy(), b, kappa)[0] <= 1e-10
    c.close()


def test_nan_gauge_link(lib):
    """A NaN link: load_gauge's unitarity check rejects it; loaded without the check, every
    solve whose sources reach it reports DL_NAN and returns (FP64 and mixed precision)."""
    dims = (4, 4, 4, 4)
    U = synthetic.gauge_field(dims, eps=0.45, seed=40)
    U[1, 2, 3, 0, 2, 1, 1] = np.nan  # [T][Z][Y][X][mu][3][3]
    c = lib.Context(dims)
    with pytest.raises(lib.DlError):
        c.load_gauge(U)
    c.load_gauge(U, check_unitarity=False)
    c.set_kappa(0.12)
    b = synthetic.random_spinor(dims, seed=41, n=2)
    for prec in (0, 1):
        _, st = c.solve(to_gpu(b), lib.Params(tol=1e-10, precision=prec, batch=2), allow_fail=True)
        assert all(s["status"] == lib.NAN for s in st), st
    c.close()


@pytest.mark.parametrize("prec, kind", [(0, 0), (1, 0), (1, 7)])
def test_skipping_stopped_rhs_changes_nothing(lib, prec, kind, monkeypatch):
    """The direct hops skip the loads and stores of right-hand sides that have stopped; the
    others' arithmetic is untouched and a stopped one's vectors stay frozen either way, so the
    solutions are bitwise the same with the skip switched off (DLOOPS_HOP_SKIP=0).  Point sources
    and Z2 sources in one batch stop at different iterations."""
    dims, kappa = (4, 4, 4, 8), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=12)
    sols = {}
    plain_f32_layout(monkeypatch, prec, kind)
    for flag in ("1", "0"):
        monkeypatch.setenv("DLOOPS_HOP_SKIP", flag)
        c = lib.Context(dims)
        c.load_gauge(U)
        c.set_kappa(kappa)
        # one fixed launch shape for both contexts: the reductions' summation order follows it
        c.tune_hop(prec, 16, force_R=2 if kind == 7 else 1, force_block=64, force_pf=kind)
        b = torch.cat([c.make_point_sources(12 * 37, 8), c.make_sources(seed=6, noise_first=0, n_noise=8,
                                                                          dilution=0)]).contiguous()
        x, st = c.solve(b, lib.Params(tol=1e-11, precision=prec, batch=16))
        assert all(s["status"] == 0 for s in st), st
        sols[flag] = (x.cpu().numpy(), [s["iters"] for s in st])
        c.close()
    monkeypatch.delenv("DLOOPS_HOP_SKIP")
    assert np.array_equal(sols["1"][0], sols["0"][0])
    assert sols["1"][1] == sols["0"][1]
    assert len(set(sols["1"][1])) > 1  # the batch really held right-hand sides that stopped early


def test_plain_and_fused_hops_on_different_kernels(lib):
    """The plain and the two fused hops take their launch shapes separately: a solve with the direct
    kernel for the plain hops, the wider-cap direct one for <rhat, v> and the warp-staged one for the
    five-reduction hop reaches the tolerance, and shapes a width cannot run are refused."""
    dims, kappa = (8, 8, 8, 24), 0.12
    U = synthetic.gauge_field(dims, eps=0.45, seed=13)
    c = lib.Context(dims)
    c.load_gauge(U)
    c.set_kappa(kappa)
    b = synthetic.random_spinor(dims, seed=23, n=32)
    c.set_hop_shape(1, 32, 0, 1, 128, 0)
    c.set_hop_shape(1, 32, 1, 1, 64, 10)
    c.set_hop_shape(1, 32, 2, 1, 64, 4)
    assert [c.hop_shape(1, 32, k) for k in (0, 1, 2)] == [(1, 128, 0), (1, 64, 10), (1, 64, 4)]
    x, st = c.solve(to_gpu(b), lib.Params(tol=1e-11, precision=1, batch=32))
    assert all(s["status"] == 0 for s in st), st
    res = residual(U, x.cpu().numpy()[[0, 31]], b[[0, 31]], kappa)
    assert np.all(res <= 1e-11), res
    for bad in ((1, 128, 4), (2, 64, 4), (1, 64, 5), (1, 64, 7), (3, 64, 0), (1, 96, 0), (2, 64, 10)):
        with pytest.raises(lib.DlError):
            c.set_hop_shape(1, 32, 2, *bad)
    with pytest.raises(lib.DlError):
        c.set_hop_shape(1, 32, 3, 1, 64, 0)
    c.close()
