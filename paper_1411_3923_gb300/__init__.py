"""GB300-native two-level spectral-MsFEM flexible CG for robust SIMP topology optimisation
of fully resolved microstructures (Alexandersen & Lazarov, arXiv:1411.3923).

The compute path is the CUDA library built from ``csrc/`` into ``_lib/libmstopo.so`` with
the C ABI of ``include/mstopo.h``; ``mstopo`` is its Python binding.
"""
from .mstopo import (FIELD_RHO_BAR, FIELD_RHO_TILDE, FIELD_YOUNG, FP64, MIXED, MMA, MstopoError,
                     PDEFilter, Problem, RobustCompliance, SYMBOLS, batch_build_preconditioner,
                     batch_solve, load)

__all__ = ["Problem", "PDEFilter", "MMA", "RobustCompliance", "MstopoError", "load", "FP64", "MIXED",
           "FIELD_RHO_TILDE", "FIELD_RHO_BAR", "FIELD_YOUNG", "SYMBOLS",
           "batch_build_preconditioner", "batch_solve"]
