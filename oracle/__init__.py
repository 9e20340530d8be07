"""Plain CPU oracle for tensor-network robust control (arXiv 2603.03639).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it; the two meet only in the
seeded inputs of ``synth``.

Everything is complex128 / float64 NumPy with LAPACK (``numpy.linalg``) as the
only library primitive, written for a reader who checks it against the paper:

  * ``noise``   -- J_b^(s) ~ U[-dJ, dJ] (Sec. II) or N(0, s^2), drawn from the
                   published counter-based SplitMix64 generator.
  * ``gates``   -- the two-site bond Hamiltonians of Eq. sysH (ZZ crosstalk
                   only) and their exact exponentials, with the Daleckii-Krein
                   derivative of the exponential for the gradient.
  * ``mps``     -- MPS canonical form, the TEBD two-site update with truncated
                   SVD (Sec. II, Eq. circuit), overlaps and mixed two-site
                   densities.
  * ``robust``  -- the ensemble-averaged fidelity (Sec. II, state form) and
                   its costate gradient (App. A), one trajectory at a time.
  * ``dense``   -- a dense state-vector propagator of the same gate sequence
                   (N <= 12) and an exact per-slice exponential.
  * ``runner``  -- a process-pool map of trajectories (the timed CPU baseline).

Parity status: every function is pinned by the ``-m "not gpu"`` tests except
the truncated regime (bond dimension capped below the exact value), where no
independent pin exists: there the oracle is the algorithm itself (parity
unpinned beyond convergence in chi).
"""
