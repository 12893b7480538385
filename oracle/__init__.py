"""Plain, slow FP64 CPU oracle of randomized resolvent analysis.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it, and it shares no code with the CUDA path: the
operator is assembled here from Kronecker products of 1-D difference
matrices (the CUDA path evaluates a per-node stencil), the factorisation is a
dense or banded LAPACK LU (the CUDA path uses a block Gauss-Jordan inverse),
QR is Householder (the CUDA path uses CholeskyQR2) and the small SVD is
LAPACK's (the CUDA path uses one-sided Jacobi).

Modules
  operator   -- the linearised operator L (Dirichlet or Neumann closure) and
                the sketch weight Phi
  philox     -- Philox-4x32-10 counter-based generator and the test-matrix
                entries (Gaussian, Rademacher, sparse Rademacher)
  resolvent  -- exact resolvent SVD, Algorithm 1 step by step, subspace
                iterations
  gradient   -- gradient of the summed leading gains with respect to the base
                flow

Functions whose results are pinned only against the paper's statements and
not against closed forms are marked "parity unpinned" in their docstrings.
"""
