"""GB300-native randomized resolvent analysis (arXiv:1902.01458).

The compute path is the CUDA library librr.so (C ABI in include/rr.h); this
package holds its sources (csrc/), the in-tree build (build.py) and a thin
ctypes binding (_lib.py).  Importing the package does not load the library;
the first call that needs it does, and fails loudly if it has not been built.
"""
from ._lib import (Batch, Factors, Operator, RRError, ResolventResult, load,  # noqa: F401
                   rr_apply, rr_create_operator, rr_destroy_factors,
                   rr_destroy_operator, rr_factor, rr_gaussian, rr_modes, rr_operator_dims,
                   rr_phi, rr_sketch, rr_solve, rr_test_matrix)
