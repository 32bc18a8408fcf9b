"""GB300 (sm_103a) RBF-FD stencil weights: kNN stencils, PHS + monomial
weights (FP64, FP32 + FP64 refinement), CSR operator application.

The compute lives in libmm.so (CUDA kernels behind the C ABI of
include/mm.h); ``binding`` is a thin ctypes layer over it.
"""
from . import _build  # noqa: F401
from .binding import (DN, DX, DY, DZ, FP32_IR, FP64, KNN_AUTO, KNN_BRUTE, KNN_GRID, LAP,  # noqa: F401
                      MLP, Context, MMError, load, rbffd_weights_surrogate, stencil_features)
