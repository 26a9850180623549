"""GB300-native Krylov-regularization solvers for MQ-RBF Helmholtz collocation.

The compute lives in ``_lib/librbfkr.so`` (CUDA for sm_103a, C ABI in
``include/rbfkr.h``); ``rbfkr`` is its thin ctypes binding and ``pipeline``
chains the entry points for one solve.  PyTorch provides device memory and
streams only.
"""
from . import rbfkr  # noqa: F401
from .rbfkr import (  # noqa: F401
    RBF_ASSEMBLED, RBF_FIXED, RBF_FORM_C, RBF_FORM_EPS, RBF_FP64, RBF_GCV, RBF_LCURVE,
    RBF_MATRIX_FREE, RBF_MIXED, Context, RbfError, load, make_state,
)
