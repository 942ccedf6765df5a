"""The allocation-free loop contraction agrees with dl_trace_loops (GPU).

dl_trace_loops_noalloc serves callers that cannot call cudaMalloc (for
example code running during CUDA-graph stream capture, or programs whose
device memory belongs to their own allocator).  It keeps its partial sums in
a fixed static device array shared by all calls.  Two calls in a row, with
different inputs, must each match the context-based contraction, which shows
the shared array carries nothing over from one call to the next.  This file
is collected last.
"""

import ctypes

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_trace_loops_twice(lib):
    dims = (4, 4, 2, 6)
    c = lib.Context(dims)
    c.load_gauge(synthetic.gauge_field(dims, eps=0.45, seed=1))
    for call, (seed, n, t_range) in enumerate([(1, 5, (0, 6)), (2, 3, (2, 5))]):
        eta = torch.from_numpy(synthetic.random_spinor(dims, seed=seed, n=n)).cuda()
        phi = torch.from_numpy(synthetic.random_spinor(dims, seed=seed + 10, n=n)).cuda()
        out = torch.full((n, 16, dims[3]), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        lib.trace_loops_noalloc(eta, phi, dims, t_range=t_range, out=out)
        torch.cuda.synchronize()
        ref = c.trace_loops(eta, phi, lib.SINK_LOCAL, t_range=t_range)[:, 0]
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), f"call {call}"
    c.close()


def test_noalloc_rejects_oversized_request(lib):
    dims = (2, 2, 2, 2)
    L = lib.lib()
    rc = L.dl_trace_loops_noalloc(ctypes.c_void_p(16), ctypes.c_void_p(16), 20000, (ctypes.c_int * 4)(*dims), 0, 1,
                                  ctypes.c_void_p(16), None)
    assert rc == lib.EINVAL
    assert b"16384" in L.dl_last_error()
