"""GB300-native space-time Ripley's K: edge-corrected K / L over a threshold grid and Monte
Carlo CSR simulation envelopes (Wang et al., Section 3), computed by hand-written CUDA kernels
behind the C ABI in include/stk.h.  This package is the thin Python binding."""
from ._lib import (  # noqa: F401
    LIB_PATH,
    STK_EDGE_ISOTROPIC,
    STK_EDGE_NONE,
    STK_EXEC_BATCHED,
    STK_EXEC_PLAIN,
    STK_NORM_N2,
    STK_NORM_N_NM1,
    STK_PREC_FP32_GUARDED,
    STK_PREC_FP64,
    Pattern,
    StkError,
    load,
    stk_create,
    stk_create_device,
    stk_destroy,
    stk_envelope,
    stk_k,
    stk_k_noalloc,
    stk_last_error,
    stk_last_stats,
    stk_run,
    stk_set_stream,
    stk_sim_points,
    stk_version,
)
