"""GB300 (sm_103a) RBF-FD stencil weights: kNN stencils, PHS + monomial
weights (FP64, FP32 inverse + refinement) of the Laplacian, first and second
derivatives and d/dn, weighted least squares (GWLS) weights, CSR operator
application, the learned surrogate.

The compute lives in libmm.so (CUDA kernels behind the C ABI of
include/mm.h); ``binding`` is a thin ctypes layer over it.
"""
from . import _build  # noqa: F401
from .binding import (DN, DX, DXX, DXY, DXZ, DY, DYY, DYZ, DZ, DZZ, FP32_IR, FP64, KNN_AUTO,  # noqa: F401
                      KNN_BRUTE, KNN_GRID, LAP, MLP, SCALE_FARTHEST, SCALE_NEAREST, Context, MMError,
                      load, partition_halo, partition_morton, rbffd_weights_surrogate,
                      stencil_features)
