"""GB300-native Sparse Gauss-Newton (SGN) for equilibrium-constrained design.

The hot path (element kernels, no-atomic assembly into the fixed pattern of
the saddle-point matrix of Eq. sparseSystemGN, multifrontal Bunch-Kaufman
LDL^T, triangular solves, FP64 refinement, Newton equilibrium and the adjoint
gradient) lives in the CUDA library ``libsgn.so`` behind the C ABI in
``include/sgn.h``.  ``SGN`` is its Python front end; ``WarmStart`` drives the
learned warm start of the equilibrium solve (``include/sgn_learn.h``).
"""
from .binding import (FP64, MIXED, RHS_KKT, RHS_PAPER, STORE_FP64, STORE_KFACT, STORE_KFACT_MIXED, STORE_MIXED,
                      SGNError, load_library)
from .learner import WarmStart
from .solver import SGN

__all__ = ["SGN", "WarmStart", "SGNError", "FP64", "MIXED", "RHS_KKT", "RHS_PAPER", "STORE_FP64", "STORE_MIXED",
           "STORE_KFACT", "STORE_KFACT_MIXED", "load_library"]
