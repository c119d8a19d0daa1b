"""GB300 (sm_103a) aggregation-AMG solver for graph Laplacians.

Flexible CG preconditioned by the nonlinear AMLI cycle (K-cycle) over
unsmoothed matching-based aggregation, with the polynomial smoother of best
uniform approximation to 1/x (Brannick, "Aggregation-based aggressive
coarsening with polynomial smoothing").  The computation lives in the CUDA
library libamg_gb300.so behind the C ABI of include/amg.h; this package only
builds it and marshals arguments (see :mod:`.binding`).
"""
from .binding import (  # noqa: F401
    AMG_AGG_MATCHING, AMG_AGG_MIS, AMG_CYCLE_AMLI, AMG_CYCLE_K, AMG_ERR_BAD_WEIGHT, AMG_ERR_BREAKDOWN,
    AMG_ERR_CUDA, AMG_ERR_DISCONNECTED, AMG_ERR_INVALID_ARG, AMG_ERR_NOT_CONVERGED,
    AMG_ERR_NOT_SYMMETRIC, AMG_ERR_OOM, AMG_ERR_SELF_LOOP, AMG_ERR_SETUP_STALL, AMG_ERR_TIMEOUT,
    AMG_MEM_DEVICE, AMG_MEM_HOST, AMG_OK, AMG_PREC_FP32, AMG_PREC_FP64, AmgError, Hierarchy,
    SYMBOLS, Server,
    amg_default_options, amg_degree_for, amg_free, amg_info, amg_last_error, amg_match,
    amg_match_noalloc, amg_options, amg_server_config, amg_server_stats_t, amg_setup, amg_solve,
    lib, library_path,
)
