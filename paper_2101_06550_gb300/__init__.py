"""GB300-native semi-implicit ADI Cahn-Hilliard stepping and batched cyclic band solvers.

The compute path is ``libchx.so`` (hand-written CUDA for sm_103a behind the C
ABI of ``include/chx.h``); this package is its thin Python binding.
"""
from ._chx import (COEF_PER_SYSTEM, COEF_SHARED, COEF_UNIFORM, EXPORTS, F32, F64, PREC_F32_REFINE, PREC_F64,
                   CN1DPlan, Ch1DPlan, ChPlan, ChxError, Ensemble, PentaPlan, TriPlan, coarsening_rate, fp64_fma_rate, lib,
                   noise_normals, stencil_apply_2d, status_string, version)

__all__ = ["ChPlan", "Ch1DPlan", "CN1DPlan", "Ensemble", "PentaPlan", "TriPlan", "ChxError", "stencil_apply_2d", "noise_normals", "coarsening_rate", "fp64_fma_rate", "lib", "status_string", "version",
           "F64", "F32", "COEF_UNIFORM", "COEF_SHARED", "COEF_PER_SYSTEM", "PREC_F64", "PREC_F32_REFINE", "EXPORTS"]
