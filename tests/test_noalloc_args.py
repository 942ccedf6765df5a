"""The binding of the allocation-free contraction rejects bad tensors before any launch (CPU).

Its kernels index eta, phi and out from n, V and T alone, so every mismatch
must be caught on the host; each case here raises before the library is called.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1012_5168_gb300 as dl

DIMS = (2, 2, 2, 4)
V = 32


def field(n, dtype=torch.complex128):
    return torch.zeros(n * V * 12, dtype=dtype)


@pytest.mark.parametrize("case, exc, text", [
    ("eta complex64", TypeError, "complex128"),
    ("phi float64", TypeError, "complex128"),
    ("eta strided", ValueError, "contiguous"),
    ("eta ragged", ValueError, "multiple of 12 V"),
    ("phi shorter", ValueError, "phi holds"),
    ("out wrong shape", ValueError, "shape"),
    ("out wrong dtype", TypeError, "out must be"),
    ("bad range", ValueError, "timeslice range"),
    ("bad dims", ValueError, "four positive"),
    ("on the host", ValueError, "CUDA tensor"),
])
def test_bad_noalloc_arguments_raise(case, exc, text):
    eta, phi, out, dims, tr = field(3), field(3), torch.zeros((3, 16, 4), dtype=torch.complex128), DIMS, None
    if case == "eta complex64":
        eta = field(3, torch.complex64)
    elif case == "phi float64":
        phi = torch.zeros(3 * V * 12, dtype=torch.float64)
    elif case == "eta strided":
        eta = torch.zeros(2 * 3 * V * 12, dtype=torch.complex128)[::2]
    elif case == "eta ragged":
        eta = torch.zeros(3 * V * 12 + 5, dtype=torch.complex128)
    elif case == "phi shorter":
        phi = field(2)
    elif case == "out wrong shape":
        out = torch.zeros((3, 16, 3), dtype=torch.complex128)
    elif case == "out wrong dtype":
        out = torch.zeros((3, 16, 4), dtype=torch.complex64)
    elif case == "bad range":
        tr = (2, 2)
    elif case == "bad dims":
        dims = (2, 2, 0, 4)
    with pytest.raises(exc, match=text):
        dl.trace_loops_noalloc(eta, phi, dims, t_range=tr, out=out)


def test_good_host_tensors_fail_only_the_device_check():
    """Well-formed tensors pass every check up to the last one, which asks for CUDA tensors."""
    with pytest.raises(ValueError, match="eta must be a CUDA tensor"):
        dl._noalloc_args(field(3), field(3), DIMS, (1, 3), torch.zeros((3, 16, 4), dtype=torch.complex128))
