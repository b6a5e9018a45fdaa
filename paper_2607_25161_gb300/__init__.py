"""GB300-native (sm_103a) fast Stokesian dynamics for rigid multi-bead
aggregates: the per-time-step saddle-point solve behind a C ABI
(include/fsd.h), with a thin ctypes binding.

The CUDA library is loaded on first use; if it is missing, every entry point
raises (there is no CPU fallback)."""

from ._binding import (  # noqa: F401
    EXPORTS, FSD_DRIFT_FIXMAN, FSD_DRIFT_RFD, FSD_EINVAL, FSD_FLAG_AUTOTUNE, FSD_FLAG_COMOVING, FSD_FLAG_GRAPH, FSD_FLAG_LEES_EDWARDS, FSD_FLAG_FP32_KRYLOV, FSD_NF_LANCZOS, FSD_NF_PAIRWISE, Batch, FSD_ENOCONV, FSD_ENUMERIC, FSD_EOVERLAP, FSD_FLAG_WARM_START, FSD_FP64,
    FSD_MIXED, FSD_OK, FsdError, FsdParams, FsdStats, Suspension, default_params, fma_throughput, load,
)
