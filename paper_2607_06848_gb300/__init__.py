"""GB300-native orthogonalized enriched finite element (EFE) Kohn-Sham eigensolver.

The compute path is the CUDA library libefe.so (C ABI in include/efe.h);
``efe`` is its ctypes binding and ``build`` compiles it in-tree for sm_103a.
"""
from .efe import (EFE, MLP, EFEError, load, EFE_FP64, EFE_FP32, EFE_BF16,  # noqa: F401
                  EFE_FILTER_RESIDUAL, EFE_FILTER_STANDARD, EFE_FILTER_KEEP_PRECISION)
