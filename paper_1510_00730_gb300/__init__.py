"""GB300-native evaluation of large multideterminant QMC wavefunctions.

The compute path lives in the CUDA library libmdet.so (C ABI in
include/mdet.h); this package only marshals arguments to it. Importing the
package does not need a GPU; evaluating does, and fails loudly when the
library or the device is missing.
"""
from .binding import (Batch, Context, MdetError, batch_evaluate, PRECISION_FP64, PRECISION_MIXED, WS_ESCALATED, WS_FALLBACK, WS_NONFINITE, WS_PSI_ZERO,
                      WS_REF_ILLCOND, WS_REF_SINGULAR, gemm_bf16, library_path, load_library, measure_fp64_rate,
                      omega_sort, truncate_norm)

__all__ = ["Batch", "batch_evaluate", "Context", "MdetError", "PRECISION_FP64", "PRECISION_MIXED", "WS_REF_SINGULAR", "WS_REF_ILLCOND",
           "WS_PSI_ZERO", "WS_NONFINITE", "WS_FALLBACK", "WS_ESCALATED", "gemm_bf16", "library_path", "load_library", "measure_fp64_rate", "omega_sort",
           "truncate_norm"]
