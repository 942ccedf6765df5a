"""Write the stored reference values under tests/golden/ using only the oracle.

Every value here is produced by the FP64 CPU oracle (never by the CUDA path):

* exact_loops_4x4x4x4.txt - L_Gamma(t) = sum_{x in t} Tr[Gamma M^{-1}(x,x)] on the
  4^4 exact-loop workload (kappa = 0.10, eps = 0.3, seed 1, antiperiodic in
  time), from the dense inverse of M; 16 Gamma x 4 timeslices, re and im.
* oracle_bicgstab_iters_16x16x16x32.txt - iterations the oracle's
  full-lattice BiCGStab needs to reach ||b - M x|| <= 1e-10 ||b|| for the first
  complex Z2 source (seed 1, noise 0) on the 16^3 x 32 workload (kappa = 0.140,
  eps = 0.45, seed 1).  The bench's CPU baseline times a few oracle iterations
  and scales by this count.

Run:  python tests/golden/make_golden.py [--skip-iters]
"""

from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402
from oracle import loops, noise, wilson  # noqa: E402


def exact_4x4x4x4():
    w = synthetic.WORKLOADS["exact_4x4x4x4"]
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    lo = loops.exact_loops_dense(U, w["kappa"], -1.0)
    path = os.path.join(HERE, "exact_loops_4x4x4x4.txt")
    with open(path, "w") as f:
        f.write("# Exact loops sum_{x in t} Tr[Gamma M^-1(x,x)] (Sec. 3, Eq. 2), 4^4 lattice,\n")
        f.write("# kappa=0.10, eps=0.3, seed=1, antiperiodic time; FP64 oracle, dense inverse.\n")
        f.write("# columns: gamma_index t re im\n")
        for g in range(16):
            for t in range(lo.shape[1]):
                f.write(f"{g} {t} {lo[g, t].real:.17e} {lo[g, t].imag:.17e}\n")
    print("wrote", path)


def iters_16x16x16x32():
    w = synthetic.WORKLOADS["wilson_16x16x16x32"]
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    b = noise.z2_noise(w["dims"], 1, 0)
    t0 = time.time()
    x, info = wilson.solve(U, b, w["kappa"], -1.0, tol=1e-10, max_iter=5000)
    dt = time.time() - t0
    path = os.path.join(HERE, "oracle_bicgstab_iters_16x16x16x32.txt")
    with open(path, "w") as f:
        f.write("# Oracle full-lattice BiCGStab (no preconditioning) on 16^3x32, kappa=0.140, eps=0.45,\n")
        f.write("# seed 1, Z2 source (seed 1, noise 0), to ||b - M x||/||b|| <= 1e-10.\n")
        f.write(f"# converged={info['converged']} true_residual={info['true_residual']:.3e} wall_s={dt:.0f}\n")
        f.write(f"{info['iters']}\n")
    print("wrote", path, info)


if __name__ == "__main__":
    exact_4x4x4x4()
    if "--skip-iters" not in sys.argv:
        iters_16x16x16x32()
