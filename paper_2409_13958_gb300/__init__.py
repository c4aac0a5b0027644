"""GB300-native periodic micromagnetic FEM effective-field library (Python binding).

The compute path is libpmfem.so (hand-written CUDA for sm_103a behind the C-ABI of
include/pmfem.h).  This package only marshals arguments: it has no CPU fallback, and
importing the binding fails loudly when the shared library is missing.
"""
from .binding import (  # noqa: F401
    PMFEM_FP64, PMFEM_FP32, PMFEM_BF16SPLIT, PMFEM_EX, PMFEM_MS, PMFEM_AP, PMFEM_AN, PMFEM_ALL,
    PMFEM_BF16_PRECORRECTION, PMFEM_BF16_PROJECTION, PMFEM_BF16_CHARGES, PMFEM_BF16_GRADIENT, PMFEM_BF16_EXCHANGE,
    PmfemError, Pmfem, PmfemBatch, load_library, SYMBOLS,
)
