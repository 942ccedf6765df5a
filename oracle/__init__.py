"""FP64 CPU oracle for the disconnected-loop hot path (test infrastructure).

This package is a plain, slow, deliberately unoptimised restatement of what the
method of "Exact calculation of disconnected loops" (Alexandrou, Christaras,
O Cais, Strelchenko, Lattice 2010) computes.  It exists only to check the CUDA
path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it; the library in
``paper_1012_5168_gb300`` never does, and the oracle imports nothing from it.

Everything is full-lattice and lexicographic (no even-odd preconditioning, no
spin projection, no batching tricks), in complex128:

* ``lattice``  - geometry, the gamma matrices and the 16-element Gamma basis;
* ``wilson``   - the Wilson hopping term D, M = 1 - kappa*D, its adjoint, the
                 dense matrix for tiny lattices, unpreconditioned BiCGStab;
* ``philox``   - the Philox4x64-10 counter-based generator (Salmon et al. 2011);
* ``noise``    - complex Z2 sources and the dilution schemes of Sec. 2;
* ``smear``    - gauge-covariant Gaussian smearing (Sec. 2);
* ``loops``    - the loop contraction Tr[Gamma S_F(x,x)] per timeslice (Sec. 3,
                 Eq. 2), exact loops from the all-to-all diagonal, the stochastic
                 estimator, the truncated-solver-method combination (Sec. 2),
                 and the adjoint-based loop gradients;
* ``correlators`` - momentum-projected loops, the disconnected correlator and
                 the connected meson correlator of a point source (Sec. 3,
                 Eqs. 1 and 3);
* ``krylov``   - the even-site Schur system written with parity projectors on
                 full-lattice fields, and the fixed-iteration Krylov maps
                 (CGNR, BiCGStab) that define the truncated solver method's
                 low-precision solves.

Pinning: every function is checked by ``tests/test_oracle_*.py`` against
facts that do not come from the oracle itself (closed forms, a dense LAPACK
inverse, numpy's least-squares solver, the hopping expansion, gauge
invariance, gamma5-hermiticity, numpy's Philox implementation).  The one piece
without such a pin is noted in ``loops.tsm_estimate``: the BF16 low-precision
solver map is parity unpinned beyond an error bound.  Its FP64 counterpart
(``krylov``) and the combination itself are pinned.
"""

from . import lattice, wilson, philox, noise, smear, loops, krylov, correlators  # noqa: F401
