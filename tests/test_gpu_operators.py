"""CUDA path vs oracle: Wilson hop, M, smearing, sources, Gamma weights (GPU).

FP64 kernels are compared element by element with the FP64 oracle; the only
difference is the order of floating-point additions, so the bound is a few
hundred ulps of the largest entry (1e-13 relative).  Integer work (noise
signs, dilution classes, point sources) must be bit-exact.
"""

import numpy as np
import pytest

import synthetic
from oracle import lattice, noise, smear, wilson

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 8), (4, 2, 6, 4)]


def ctx_for(dl, dims, kappa=0.13, eps=0.45, seed=5, t_bc=-1):
    U = synthetic.gauge_field(dims, eps=eps, seed=seed)
    c = dl.Context(dims, t_bc=t_bc)
    c.load_gauge(U)
    c.set_kappa(kappa)
    return c, U


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_hop_matches_oracle(lib, dims, t_bc):
    c, U = ctx_for(lib, dims, t_bc=t_bc)
    psi = synthetic.random_spinor(dims, seed=1, n=3)
    out = c.apply_hop(to_gpu(psi)).cpu().numpy()
    ref = wilson.hop(U, psi, float(t_bc))
    assert rel(out, ref) < 1e-13
    m = c.apply_m(to_gpu(psi)).cpu().numpy()
    assert rel(m, wilson.apply_m(U, psi, 0.13, float(t_bc))) < 1e-13
    c.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8)])
def test_float_float_hop_matches_oracle(lib, dims, monkeypatch):
    """The float-float hop of the defect-correction steps: about 48 significant bits.

    Inputs span magnitudes from 1e-20 to 1e3 with zeros, so the bit-level
    double -> float-float split is exercised over many exponents.
    """
    c, U = ctx_for(lib, dims)
    psi = synthetic.random_spinor(dims, seed=11, n=3)
    rng = np.random.default_rng(3)
    psi[1] *= 10.0 ** rng.uniform(-20, 3, size=psi[1].shape)
    psi[2].reshape(-1)[::7] = 0.0
    monkeypatch.setenv("DLOOPS_HOP_ARITH", "dff")
    out = c.apply_hop(to_gpu(psi)).cpu().numpy()
    m = c.apply_m(to_gpu(psi)).cpu().numpy()
    monkeypatch.delenv("DLOOPS_HOP_ARITH")
    for j in range(3):
        ref = wilson.hop(U, psi[j:j + 1], -1.0)
        assert np.linalg.norm(out[j:j + 1] - ref) < 2e-14 * np.linalg.norm(ref)
        refm = wilson.apply_m(U, psi[j:j + 1], 0.13, -1.0)
        assert np.linalg.norm(m[j:j + 1] - refm) < 2e-14 * np.linalg.norm(refm)
    c.close()


def test_hop_full_size(lib):
    dims = (16, 16, 16, 32)
    c, U = ctx_for(lib, dims, kappa=0.14, seed=1)
    psi = synthetic.random_spinor(dims, seed=2, n=1)
    out = c.apply_hop(to_gpu(psi)).cpu().numpy()
    assert rel(out, wilson.hop(U, psi, -1.0)) < 1e-13
    c.close()


@pytest.mark.parametrize("dil", [
    0, noise.SPIN, noise.SPIN | noise.COLOUR, noise.SPIN | noise.COLOUR | noise.EVENODD | noise.TIME,
    noise.CUBIC, noise.COLOUR | noise.CUBIC | noise.TIME, noise.EVENODD | noise.CUBIC,
])
def test_sources_bit_exact(lib, dil):
    dims = (4, 4, 2, 6)
    c, _ = ctx_for(lib, dims)
    for t0 in (-1, 3):
        got = c.make_sources(seed=2**63 + 11, noise_first=5, n_noise=3, dilution=dil, t0=t0).cpu().numpy()
        ref = noise.make_sources(dims, 2**63 + 11, 5, 3, dil, t0=t0)
        assert np.array_equal(got, ref)
    c.close()


def test_sources_full_size_bit_exact(lib):
    dims = (16, 16, 16, 32)
    c, _ = ctx_for(lib, dims)
    got = c.make_sources(seed=1, noise_first=63, n_noise=1, dilution=0, t0=0).cpu().numpy()
    assert np.array_equal(got[0], noise.z2_noise(dims, 1, 63))
    c.close()


def test_point_sources(lib):
    dims = (2, 2, 2, 4)
    c, _ = ctx_for(lib, dims)
    got = c.make_point_sources(17, 40).cpu().numpy()
    ref = noise.point_sources(dims, 17, 40)
    assert np.array_equal(got, ref)
    assert np.array_equal(c.make_point_sources(17, 40, prec=lib.PREC_F32).cpu().numpy(), ref.astype(np.complex64))
    bf = c.make_point_sources(17, 40, prec=lib.PREC_BF16).float().cpu().numpy()
    assert np.array_equal(bf[..., 0] + 1j * bf[..., 1], ref)
    c.close()


def bf16_round(x: np.ndarray) -> np.ndarray:
    """float64 -> float32 (nearest) -> bfloat16 (nearest, ties to even), returned as float32."""
    f = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("dil", [0, 1 | 2 | 4 | 16])
def test_sources_in_working_precision(lib, dil):
    """complex64 and bfloat16 sources are the oracle's complex128 values rounded to nearest."""
    dims = (4, 4, 2, 6)
    c, _ = ctx_for(lib, dims)
    ref = noise.make_sources(dims, 77, 2, 3, dil, t0=-1)
    f32 = c.make_sources(seed=77, noise_first=2, n_noise=3, dilution=dil, t0=-1, prec=lib.PREC_F32).cpu().numpy()
    assert f32.dtype == np.complex64 and np.array_equal(f32, ref.astype(np.complex64))
    bf = c.make_sources(seed=77, noise_first=2, n_noise=3, dilution=dil, t0=-1, prec=lib.PREC_BF16)
    bf = bf.float().cpu().numpy()
    assert np.array_equal(bf[..., 0], bf16_round(ref.real)) and np.array_equal(bf[..., 1], bf16_round(ref.imag))
    assert set(np.unique(np.abs(bf))) <= {0.0, float(bf16_round(np.array([np.sqrt(0.5)]))[0])}
    c.close()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 2)])
def test_smearing_matches_oracle(lib, dims):
    c, U = ctx_for(lib, dims)
    psi = synthetic.random_spinor(dims, seed=3, n=3)
    out = c.apply_smear(to_gpu(psi), 4.0, 7).cpu().numpy()
    assert rel(out, smear.smear(U, psi, 4.0, 7)) < 1e-13
    # timeslice restriction: other timeslices zero, the range exact
    out = c.apply_smear(to_gpu(psi), 2.5, 5, t_range=(1, 2)).cpu().numpy()
    ref = smear.smear(U, psi, 2.5, 5)
    assert np.all(out[:, 0] == 0) and rel(out[:, 1], ref[:, 1]) < 1e-13
    c.close()


def test_gamma_weights(lib):
    dims = (2, 2, 2, 4)
    c, _ = ctx_for(lib, dims)
    psi = synthetic.random_spinor(dims, seed=4, n=2)
    rng = np.random.default_rng(0)
    w = rng.standard_normal((2, 16, 4)) + 1j * rng.standard_normal((2, 16, 4))
    gb = lattice.gamma_basis()
    for mode in (0, 1):
        out = c.apply_gamma_weights(to_gpu(psi), w, mode).cpu().numpy()
        ref = np.zeros_like(psi)
        for j in range(2):
            for t in range(4):
                m = sum((w[j, g, t] * gb[g].conj().T) if mode == 0 else (np.conj(w[j, g, t]) * gb[g]) for g in range(16))
                ref[j, t] = np.einsum("sr,...ra->...sa", m, psi[j, t])
        assert rel(out, ref) < 1e-14
    c.close()


def test_bad_inputs_rejected(lib):
    dims = (4, 4, 4, 4)
    c = lib.Context(dims)
    U = synthetic.gauge_field(dims, eps=0.3, seed=1)
    U[0, 0, 0, 0, 0, 0, 0] *= 1.5
    with pytest.raises(lib.DlError) as e:
        c.load_gauge(U)
    assert e.value.status == lib.EINVAL
    x = torch.zeros((1, 4, 4, 4, 4, 4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(lib.DlError) as e:
        c.solve(x)
    assert e.value.status == lib.ESTATE
    c.close()


def test_fma_rate_measured(lib):
    """The FMA microbenchmark returns a positive rate, FP32 above FP64, and rejects other precisions."""
    f64, ms64 = lib.bench_fma(lib.PREC_F64)
    f32, ms32 = lib.bench_fma(lib.PREC_F32)
    assert f64 > 0 and ms64 > 0 and f32 > f64
    with pytest.raises(lib.DlError) as e:
        lib.bench_fma(lib.PREC_BF16)
    assert e.value.status == lib.EINVAL
