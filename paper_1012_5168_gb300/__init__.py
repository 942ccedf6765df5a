"""GB300 (sm_103a) disconnected quark loops: thin Python binding of ``include/dloops.h``.

The computation ("Exact calculation of disconnected loops", Lattice 2010:
repeated Wilson-Dirac inversions over point or diluted complex Z2 sources and
the loop contraction Tr[Gamma M^{-1}(x, x)] per timeslice, Sec. 2-3) runs in
the CUDA kernels of ``libdloops.so``.  This module only marshals arguments:
torch tensors supply device memory and the current CUDA stream, numpy arrays
the host gauge field; every call forwards to the C ABI of the same name.

Field tensors are complex128 CUDA tensors whose memory holds the canonical
layout ``[n_rhs][V][4 spin][3 colour]`` (for instance shaped
``(n, T, Lz, Ly, Lx, 4, 3)``, the same order as the numpy arrays of the
``synthetic`` inputs).  There is no CPU fallback: without the built library
or a CUDA device every call raises.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdloops.so")

# enums of dloops.h
OK, EINVAL, ENOMEM, ECUDA, NOT_CONVERGED, BREAKDOWN, NAN, ESTATE = range(8)
PREC_F64, PREC_F32, PREC_BF16 = 0, 1, 2
METHOD_BICGSTAB, METHOD_CGNR = 0, 1
DIL_SPIN, DIL_COLOUR, DIL_EVENODD, DIL_CUBIC, DIL_TIME = 1, 2, 4, 8, 16
SINK_LOCAL, SINK_SMEARED, SUM_T = 1, 2, 4

GAMMA_NAMES = ("1", "g1", "g2", "g3", "g4", "g5", "g5g1", "g5g2", "g5g3", "g5g4",
               "g1g2", "g1g3", "g1g4", "g2g3", "g2g4", "g3g4")

# every entry point of the C ABI, as declared in include/dloops.h
SYMBOLS = (
    "dl_create", "dl_destroy", "dl_last_error", "dl_status_string", "dl_load_gauge", "dl_set_kappa", "dl_set_clover",
    "dl_set_timing", "dl_get_timing", "dl_make_sources", "dl_make_point_sources", "dl_solve",
    "dl_solve_adjoint", "dl_apply_hop", "dl_apply_m", "dl_apply_dm_dkappa", "dl_apply_clover", "dl_apply_smear", "dl_apply_gamma_weights",
    "dl_trace_loops", "dl_exact_loops", "dl_tsm_estimate", "dl_bench_hop", "dl_tune_hop", "dl_hop_shape", "dl_set_hop_shape",
    "dl_trace_loops_noalloc", "dl_bench_fma", "dl_trace_loops_mom", "dl_meson_correlators", "dl_disconnected",
    "dl_apply_hop_prec", "dl_dilution_error",
)


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("precision", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("fixed_iters", ctypes.c_int), ("delta", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("batch", ctypes.c_int), ("use_graph", ctypes.c_int), ("chunk", ctypes.c_int),
                ("method", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer", ctypes.c_int),
                ("true_residual", ctypes.c_double)]


class Smear(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("n_iter", ctypes.c_int)]


class Timing(ctypes.Structure):
    _fields_ = [("hop_ms", ctypes.c_double * 4), ("hop_launches", ctypes.c_int64 * 4),
                ("hop_bytes", ctypes.c_double * 4), ("kernel_launches", ctypes.c_int64)]


class DlError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"dloops error {status}: {message}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """Load libdloops.so (built in-tree by ``paper_1012_5168_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1012_5168_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, d, u64, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "dl_create": (i, [P(vp), P(i), i, vp]),
        "dl_destroy": (i, [vp]),
        "dl_last_error": (ctypes.c_char_p, []),
        "dl_status_string": (ctypes.c_char_p, [i]),
        "dl_load_gauge": (i, [vp, vp, i]),
        "dl_set_kappa": (i, [vp, d]),
        "dl_set_clover": (i, [vp, d]),
        "dl_set_timing": (i, [vp, i]),
        "dl_get_timing": (i, [vp, P(Timing), i]),
        "dl_make_sources": (i, [vp, u64, i64, i, ctypes.c_uint, i, i, vp, P(i64)]),
        "dl_make_point_sources": (i, [vp, i64, i, i, vp]),
        "dl_solve": (i, [vp, vp, vp, i, P(SolveParams), P(SolveStats)]),
        "dl_solve_adjoint": (i, [vp, vp, vp, i, P(SolveParams), P(SolveStats)]),
        "dl_apply_hop": (i, [vp, vp, vp, i]),
        "dl_apply_hop_prec": (i, [vp, i, vp, vp, i]),
        "dl_dilution_error": (i, [vp, u64, i, ctypes.c_uint, i, P(SolveParams), vp, vp, vp]),
        "dl_apply_m": (i, [vp, vp, vp, i]),
        "dl_apply_dm_dkappa": (i, [vp, vp, vp, i]),
        "dl_apply_clover": (i, [vp, vp, vp, i, i]),
        "dl_apply_smear": (i, [vp, vp, vp, i, P(Smear), i, i]),
        "dl_apply_gamma_weights": (i, [vp, vp, vp, i, vp, i, i]),
        "dl_trace_loops": (i, [vp, vp, vp, i, i, P(Smear), i, i, P(i), i, vp]),
        "dl_exact_loops": (i, [vp, i64, i64, P(SolveParams), i, P(Smear), vp, P(SolveStats)]),
        "dl_tsm_estimate": (i, [vp, u64, i, i, ctypes.c_uint, i, P(SolveParams), P(SolveParams), i, P(Smear),
                                vp, vp, vp]),
        "dl_bench_hop": (i, [vp, i, i, i, i, P(d), P(d)]),
        "dl_tune_hop": (i, [vp, i, i, i, i, i, P(i), P(i), P(i), P(d)]),
        "dl_hop_shape": (i, [vp, i, i, i, P(i), P(i), P(i)]),
        "dl_set_hop_shape": (i, [vp, i, i, i, i, i, i]),
        "dl_trace_loops_noalloc": (i, [vp, vp, i, P(i), i, i, vp, vp]),
        "dl_bench_fma": (i, [i, vp, P(d), P(d)]),
        "dl_trace_loops_mom": (i, [vp, vp, vp, i, i, P(Smear), P(i), i, P(i), i, vp]),
        "dl_meson_correlators": (i, [vp, vp, P(i), P(i), i, vp]),
        "dl_disconnected": (i, [vp, vp, vp, i, P(i), i, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, allow=()):
    if status != OK and status not in allow:
        msg = lib().dl_last_error().decode()
        raise DlError(status, msg)
    return status


@dataclass
class Params:
    """Solver parameters (dl_solve_params)."""
    tol: float = 1e-10
    precision: int = PREC_F32
    max_iter: int = 20000
    fixed_iters: int = 0
    delta: float = 0.0
    max_outer: int = 0
    batch: int = 16
    use_graph: int = 1
    chunk: int = 0
    method: int = 0  # METHOD_BICGSTAB or METHOD_CGNR

    def c(self) -> SolveParams:
        return SolveParams(self.tol, self.precision, self.max_iter, self.fixed_iters, self.delta,
                           self.max_outer, self.batch, self.use_graph, self.chunk, self.method)


def n_classes(dilution: int) -> int:
    """Diluted sources per noise vector for a dilution bitmask."""
    return ((4 if dilution & DIL_SPIN else 1) * (3 if dilution & DIL_COLOUR else 1)
            * (2 if dilution & DIL_EVENODD else 1) * (8 if dilution & DIL_CUBIC else 1))


def _noalloc_args(eta, phi, dims, t_range, out):
    """Check the tensors of trace_loops_noalloc before anything reaches the library:
    the kernels index the buffers from n, V and T alone, so a wrong dtype, size or
    layout would make them read or write past the end.  Returns (dims, n, lo, hi)."""
    import torch
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4 or min(dims) < 1:
        raise ValueError("dims must be four positive extents (Lx, Ly, Lz, T)")
    V = int(np.prod(dims))
    T = dims[3]
    for name, t in (("eta", eta), ("phi", phi)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.dtype != torch.complex128:
            raise TypeError(f"{name} must be complex128, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if eta.numel() % (12 * V) != 0:
        raise ValueError(f"eta holds {eta.numel()} complex values, not a multiple of 12 V = {12 * V}")
    n = eta.numel() // (12 * V)
    if phi.numel() != eta.numel():
        raise ValueError(f"phi holds {phi.numel()} complex values, eta {eta.numel()}")
    lo, hi = (0, T) if t_range is None else (int(t_range[0]), int(t_range[1]))
    if not (0 <= lo < hi <= T):
        raise ValueError(f"bad timeslice range [{lo}, {hi}) for T = {T}")
    if out is not None:
        if not isinstance(out, torch.Tensor) or out.dtype != torch.complex128 or not out.is_contiguous():
            raise TypeError("out must be a contiguous complex128 torch tensor")
        if tuple(out.shape) != (n, 16, T):
            raise ValueError(f"out must have shape {(n, 16, T)}, got {tuple(out.shape)}")
    for name, t in (("eta", eta), ("phi", phi)) + ((("out", out),) if out is not None else ()):
        if t.device.type != "cuda":
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device != eta.device:
            raise ValueError(f"{name} is on {t.device}, eta on {eta.device}")
    return dims, n, lo, hi


def trace_loops_noalloc(eta, phi, dims, t_range=None, out=None, stream=None):
    """Local loops without a context or any allocation inside the library.

    eta, phi: contiguous complex128 CUDA tensors in the canonical layout, n fields
    each; returns (or fills) a complex128 CUDA tensor [n, 16, T].  For callers
    that cannot allocate device memory: the library keeps its partial sums in
    fixed static storage (n * (t_hi - t_lo) <= 16384); pass a preallocated `out`.
    Every argument is checked here before the call (dtype, layout, sizes, device).
    """
    import torch
    dims, n, lo, hi = _noalloc_args(eta, phi, dims, t_range, out)
    if out is None:
        out = torch.empty((n, 16, dims[3]), dtype=torch.complex128, device=eta.device)
    if stream is None:
        stream = torch.cuda.current_stream(eta.device).cuda_stream
    _check(lib().dl_trace_loops_noalloc(ctypes.c_void_p(eta.data_ptr()), ctypes.c_void_p(phi.data_ptr()), n,
                                        (ctypes.c_int * 4)(*dims), lo, hi, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(stream)))
    return out


def bench_fma(precision: int, stream=None):
    """Measured FMA rate of the current GPU at PREC_F64 or PREC_F32: (TFLOP/s, kernel ms)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().dl_bench_fma(precision, ctypes.c_void_p(stream), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def _stats(arr) -> list:
    return [dict(status=s.status, iters=s.iters, outer=s.outer, true_residual=s.true_residual) for s in arr]


class Context:
    """One lattice on the current CUDA device (dl_create ... dl_destroy)."""

    def __init__(self, dims, t_bc: int = -1, stream=None):
        import torch
        self._torch = torch
        L = lib()
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        _check(L.dl_create(ctypes.byref(h), (ctypes.c_int * 4)(*self.dims), int(t_bc), ctypes.c_void_p(stream)))
        self._h = h

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().dl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- marshalling helpers ------------------------------------------------
    def _field(self, t, name="field"):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
            raise TypeError(f"{name} must be a complex128 CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() % (12 * self.V):
            raise ValueError(f"{name} has {t.numel()} elements, not a multiple of 12V = {12 * self.V}")
        return t.numel() // (12 * self.V)

    def new_fields(self, n: int):
        lx, ly, lz, lt = self.dims
        return self._torch.zeros((n, lt, lz, ly, lx, 4, 3), dtype=self._torch.complex128, device=self.device)

    # -- C ABI ------------------------------------------------------------
    def load_gauge(self, U: np.ndarray, check_unitarity: bool = True):
        U = np.ascontiguousarray(U, dtype=np.complex128)
        if U.size != self.V * 36:
            raise ValueError("gauge field must hold V*4*3*3 complex numbers")
        _check(lib().dl_load_gauge(self._h, U.ctypes.data_as(ctypes.c_void_p), int(check_unitarity)))

    def set_kappa(self, kappa: float):
        _check(lib().dl_set_kappa(self._h, float(kappa)))

    def set_clover(self, c_sw: float):
        """Clover coefficient c_sw of M = A - kappa D (0: plain Wilson, the default)."""
        _check(lib().dl_set_clover(self._h, float(c_sw)))

    def set_timing(self, enable: bool):
        _check(lib().dl_set_timing(self._h, int(enable)))

    def get_timing(self, reset: bool = False) -> dict:
        t = Timing()
        _check(lib().dl_get_timing(self._h, ctypes.byref(t), int(reset)))
        return dict(hop_ms=list(t.hop_ms), hop_launches=list(t.hop_launches), hop_bytes=list(t.hop_bytes),
                    kernel_launches=int(t.kernel_launches))

    def _source_out(self, n: int, prec: int, out, name="out"):
        """A caller-owned output of n canonical fields in the storage of `prec`: complex128
        (PREC_F64), complex64 (PREC_F32), or bfloat16 (re, im) pairs [n, T, Z, Y, X, 4, 3, 2]
        (PREC_BF16)."""
        torch = self._torch
        lx, ly, lz, lt = self.dims
        shape = (n, lt, lz, ly, lx, 4, 3)
        dtype = {PREC_F64: torch.complex128, PREC_F32: torch.complex64, PREC_BF16: torch.bfloat16}.get(prec)
        if dtype is None:
            raise ValueError(f"unknown precision {prec}")
        if prec == PREC_BF16:
            shape = shape + (2,)
        if out is None:
            return torch.empty(shape, dtype=dtype, device=self.device)
        if out.dtype != dtype or not out.is_contiguous() or out.device.type != "cuda":
            raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")
        if out.numel() < int(np.prod(shape)):
            raise ValueError(f"{name} is too small")
        return out

    def make_sources(self, seed: int, noise_first: int, n_noise: int, dilution: int, t0: int = 0, out=None,
                     prec: int = PREC_F64):
        """Diluted complex Z2 sources (n_noise * classes fields), written by the library in the
        storage of `prec` (complex128 by default; the solver takes complex128)."""
        n_rhs = n_classes(dilution) * n_noise
        if prec == PREC_F64 and out is not None and self._field(out, "out") < n_rhs:
            raise ValueError("out is too small")
        out = self._source_out(n_rhs, prec, out)
        _check(lib().dl_make_sources(self._h, seed, noise_first, n_noise, dilution, t0, int(prec),
                                     ctypes.c_void_p(out.data_ptr()), None))
        return out

    def make_point_sources(self, first: int, n: int, out=None, prec: int = PREC_F64):
        out = self._source_out(n, prec, out)
        _check(lib().dl_make_point_sources(self._h, first, n, int(prec), ctypes.c_void_p(out.data_ptr())))
        return out

    def _solve(self, fn, b, params, x, allow_fail):
        n = self._field(b, "b")
        if x is None:
            x = self._torch.empty_like(b)
        p = (params or Params()).c()
        st = (SolveStats * max(n, 1))()
        rc = fn(self._h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), n, ctypes.byref(p), st)
        _check(rc, allow=(NOT_CONVERGED, BREAKDOWN, NAN) if allow_fail else ())
        return x, _stats(st[:n])

    def solve(self, b, params: Params | None = None, x=None, allow_fail: bool = False):
        return self._solve(lib().dl_solve, b, params, x, allow_fail)

    def solve_adjoint(self, b, params: Params | None = None, x=None, allow_fail: bool = False):
        return self._solve(lib().dl_solve_adjoint, b, params, x, allow_fail)

    def apply_hop(self, x, out=None, precision: int | None = None):
        """out = D x (FP64); with precision PREC_F32 or PREC_BF16, the inner solver's
        low-precision hop on x rounded to that storage type, widened back to complex128."""
        n = self._field(x)
        out = self._torch.empty_like(x) if out is None else out
        if precision is None:
            _check(lib().dl_apply_hop(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), n))
        else:
            _check(lib().dl_apply_hop_prec(self._h, int(precision), ctypes.c_void_p(x.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), n))
        return out

    def apply_m(self, x, out=None):
        n = self._field(x)
        out = self._torch.empty_like(x) if out is None else out
        _check(lib().dl_apply_m(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), n))
        return out

    def apply_dm_dkappa(self, x, out=None):
        """-dM/dkappa x: D x, plus the clover term c_sw sum sigma F x when c_sw != 0."""
        n = self._field(x)
        out = self._torch.empty_like(x) if out is None else out
        _check(lib().dl_apply_dm_dkappa(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), n))
        return out

    def apply_clover(self, x, inverse: bool = False, out=None):
        """A x or A^-1 x (the clover blocks; the identity when c_sw = 0)."""
        n = self._field(x)
        out = self._torch.empty_like(x) if out is None else out
        _check(lib().dl_apply_clover(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), n,
                                     int(inverse)))
        return out

    def apply_smear(self, x, alpha: float, n_iter: int, t_range=None, out=None):
        n = self._field(x)
        out = self._torch.empty_like(x) if out is None else out
        lo, hi = t_range if t_range is not None else (0, self.dims[3])
        s = Smear(alpha, n_iter)
        _check(lib().dl_apply_smear(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), n,
                                    ctypes.byref(s), lo, hi))
        return out

    def apply_gamma_weights(self, x, w: np.ndarray, mode: int, out=None, accumulate: bool = False):
        """mode 0: out (+)= sum_G w[j,G,t] G^dag x ; mode 1: out (+)= sum_G conj(w[j,G,t]) G x."""
        n = self._field(x)
        w = np.ascontiguousarray(w, dtype=np.complex128)
        if w.shape != (n, 16, self.dims[3]):
            raise ValueError("weights must have shape (n_rhs, 16, T)")
        out = self._torch.zeros_like(x) if out is None else out
        _check(lib().dl_apply_gamma_weights(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            n, w.ctypes.data_as(ctypes.c_void_p), mode, int(accumulate)))
        return out

    def trace_loops(self, eta, phi, sink: int = SINK_LOCAL, smear=None, t_range=None, sum_rhs: bool = False,
                    t_of_rhs=None, group: int | None = None, sum_t: bool = False):
        """Loops sum_{x in t} eta^dag Gamma phi: complex array [n/group][n_sinks][16][T].

        t_of_rhs: optional per-pair timeslice (time-diluted sources); group: sum
        each run of `group` consecutive pairs (default 1, or n with sum_rhs);
        sum_t: the library sums the timeslices (last axis of length 1).
        """
        n = self._field(eta, "eta")
        if self._field(phi, "phi") != n:
            raise ValueError("eta and phi hold different numbers of fields")
        T = self.dims[3]
        lo, hi = t_range if t_range is not None else (0, T)
        if group is None:
            group = max(n, 1) if sum_rhs else 1
        n_sinks = (1 if sink & SINK_LOCAL else 0) + (1 if sink & SINK_SMEARED else 0)
        out = np.zeros((max(n // group, 1) if sum_rhs else n // group, n_sinks, 16, 1 if sum_t else T),
                       dtype=np.complex128)
        sm = Smear(*smear) if smear is not None else None
        tarr = None
        if t_of_rhs is not None:
            tarr = (ctypes.c_int * n)(*[int(t) for t in t_of_rhs])
        _check(lib().dl_trace_loops(self._h, ctypes.c_void_p(eta.data_ptr()), ctypes.c_void_p(phi.data_ptr()), n,
                                    sink | (SUM_T if sum_t else 0), ctypes.byref(sm) if sm is not None else None,
                                    lo, hi, tarr, group,
                                    out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def trace_loops_mom(self, eta, phi, momenta, sink: int = SINK_LOCAL, smear=None, t_of_rhs=None,
                        group: int = 1):
        """Momentum-projected loops sum_{x in t} exp(-i p.x) eta^dag Gamma phi:
        complex array [n/group][n_sinks][n_mom][16][T]; momenta: integer triples n (p = 2 pi n / L)."""
        n = self._field(eta, "eta")
        if self._field(phi, "phi") != n:
            raise ValueError("eta and phi hold different numbers of fields")
        T = self.dims[3]
        mom = np.ascontiguousarray(np.asarray(momenta, dtype=np.int32).reshape(-1, 3))
        n_sinks = (1 if sink & SINK_LOCAL else 0) + (1 if sink & SINK_SMEARED else 0)
        out = np.zeros((n // group, n_sinks, len(mom), 16, T), dtype=np.complex128)
        sm = Smear(*smear) if smear is not None else None
        tarr = (ctypes.c_int * n)(*[int(t) for t in t_of_rhs]) if t_of_rhs is not None else None
        _check(lib().dl_trace_loops_mom(self._h, ctypes.c_void_p(eta.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                                        n, sink, ctypes.byref(sm) if sm is not None else None,
                                        mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(mom), tarr, group,
                                        out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def meson_correlators(self, prop, src, momenta=((0, 0, 0),)):
        """Connected C^{BA}(p, t) of a point source: complex array [n_mom][16 A][16 B][T].
        prop: the 12 canonical solutions for the source (column 3 alpha + a)."""
        if self._field(prop, "prop") != 12:
            raise ValueError("prop must hold the 12 point-source solutions")
        T = self.dims[3]
        mom = np.ascontiguousarray(np.asarray(momenta, dtype=np.int32).reshape(-1, 3))
        out = np.zeros((len(mom), 16, 16, T), dtype=np.complex128)
        _check(lib().dl_meson_correlators(self._h, ctypes.c_void_p(prop.data_ptr()), (ctypes.c_int * 4)(*src),
                                          mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(mom),
                                          out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def disconnected(self, loops, momenta, cover=None):
        """D^{BA}(p, dt) from per-noise loops [n_noise][n_mom][16][T] (complex), over distinct noise
        pairs; cover: optional bool [n_noise][T].  Returns complex [n_mom][16 A][16 B][T]."""
        T = self.dims[3]
        L = np.ascontiguousarray(np.asarray(loops, dtype=np.complex128))
        mom = np.ascontiguousarray(np.asarray(momenta, dtype=np.int32).reshape(-1, 3))
        if L.shape[1:] != (len(mom), 16, T):
            raise ValueError("loops must be [n_noise][n_mom][16][T]")
        cv = None
        if cover is not None:
            cv = np.ascontiguousarray(np.asarray(cover, dtype=np.uint8))
        out = np.zeros((len(mom), 16, 16, T), dtype=np.complex128)
        _check(lib().dl_disconnected(self._h, L.ctypes.data_as(ctypes.c_void_p),
                                     cv.ctypes.data_as(ctypes.c_void_p) if cv is not None else None, L.shape[0],
                                     mom.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(mom),
                                     out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def exact_loops(self, src_first: int, n_src: int, params: Params | None = None, sink: int = SINK_LOCAL,
                    smear=None):
        T = self.dims[3]
        n_sinks = (1 if sink & SINK_LOCAL else 0) + (1 if sink & SINK_SMEARED else 0)
        out = np.zeros((n_sinks, 16, T), dtype=np.complex128)
        p = (params or Params()).c()
        sm = Smear(*smear) if smear is not None else None
        st = SolveStats()
        _check(lib().dl_exact_loops(self._h, src_first, n_src, ctypes.byref(p), sink,
                                    ctypes.byref(sm) if sm is not None else None,
                                    out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st)))
        return out, _stats([st])[0]

    def tsm_estimate(self, seed: int, n_lp: int, n_hp: int, dilution: int, t0: int, lp: Params, hp: Params,
                     sink: int = SINK_LOCAL, smear=None, per_noise: bool = False):
        T = self.dims[3]
        n_sinks = (1 if sink & SINK_LOCAL else 0) + (1 if sink & SINK_SMEARED else 0)
        mean = np.zeros((n_sinks, 16, T), dtype=np.complex128)
        var = np.zeros((n_sinks, 16, T), dtype=np.complex128)
        pn = np.zeros((n_lp + 2 * n_hp, n_sinks, 16, T), dtype=np.complex128) if per_noise else None
        a, b = lp.c(), hp.c()
        sm = Smear(*smear) if smear is not None else None
        _check(lib().dl_tsm_estimate(self._h, seed, n_lp, n_hp, dilution, t0, ctypes.byref(a), ctypes.byref(b), sink,
                                     ctypes.byref(sm) if sm is not None else None,
                                     mean.ctypes.data_as(ctypes.c_void_p), var.ctypes.data_as(ctypes.c_void_p),
                                     pn.ctypes.data_as(ctypes.c_void_p) if pn is not None else None))
        return (mean, var, pn) if per_noise else (mean, var)

    def dilution_error(self, seed: int, n_noise: int, dilution: int, t0: int, params: Params, exact: np.ndarray,
                       per_noise: bool = False):
        """Dilution study: per Gamma, the mean squared deviation of one noise vector's loop
        estimate from the exact loops `exact` [16][T] (dl_dilution_error).  Returns sigma2 [16]
        (and the per-noise loops [n_noise][16][T] with per_noise=True)."""
        T = self.dims[3]
        ex = np.ascontiguousarray(np.asarray(exact, dtype=np.complex128).reshape(16, T))
        sig = np.zeros(16, dtype=np.float64)
        pn = np.zeros((n_noise, 16, T), dtype=np.complex128) if per_noise else None
        p = params.c()
        rc = lib().dl_dilution_error(self._h, seed, n_noise, dilution, t0, ctypes.byref(p),
                                     ex.ctypes.data_as(ctypes.c_void_p), sig.ctypes.data_as(ctypes.c_void_p),
                                     pn.ctypes.data_as(ctypes.c_void_p) if pn is not None else None)
        _check(rc)
        return (sig, pn) if per_noise else sig

    def bench_hop(self, precision: int, n_rhs: int, fused: int = 0, reps: int = 20):
        """Time one hop kind alone (fused: 0 plain, 1 XPAY + <rhat, v>, 2 XPAY + five reductions)."""
        ms, by = ctypes.c_double(), ctypes.c_double()
        _check(lib().dl_bench_hop(self._h, precision, n_rhs, int(fused), reps, ctypes.byref(ms), ctypes.byref(by)))
        return ms.value, by.value

    def tune_hop(self, precision: int, n_rhs: int, force_R: int = 0, force_block: int = 0, force_pf: int = -1):
        """Autotune (or force) the hop launch shapes; returns the fused hop's (R, block, kind) and the ms of
        one plain plus one fused hop."""
        R, B, pf, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().dl_tune_hop(self._h, precision, n_rhs, force_R, force_block, force_pf, ctypes.byref(R),
                                 ctypes.byref(B), ctypes.byref(pf), ctypes.byref(ms)))
        return R.value, B.value, pf.value, ms.value

    def hop_shape(self, precision: int, n_rhs: int, cls: int):
        """(R, block, kind) the context uses for a class of hops of this width: 0 plain, 1 fused,
        2 fused with the five BiCGStab reductions."""
        R, B, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().dl_hop_shape(self._h, precision, n_rhs, int(cls), ctypes.byref(R), ctypes.byref(B),
                                  ctypes.byref(k)))
        return R.value, B.value, k.value

    def set_hop_shape(self, precision: int, n_rhs: int, cls: int, R: int, block: int, kind: int):
        """Pin the launch shape of a class of hops of this width (classes as hop_shape)."""
        _check(lib().dl_set_hop_shape(self._h, precision, n_rhs, int(cls), R, block, kind))
