"""trx — recursive TRSM / TRMM for NVIDIA GB300 (sm_103a).

Implements the recursive scheme of arXiv 2504.13821 (Section 3.1: split the
triangle, recurse on the diagonal blocks, GEMM-update the off-diagonal block,
small base kernels at the leaves) as hand-written CUDA behind the C ABI in
include/trx.h. This package is the thin Python binding (argument marshalling
over torch tensors); the CUDA library is built in-tree by ``build.py``.
"""
from ._binding import (  # noqa: F401
    Batch, Factor, GEMM_AUTO, GEMM_SIMT, GEMM_TC, OPT_GEMM, OPT_GRAPH, OPT_LEAF, OPT_PANELS, OPT_PDL, OPT_PROFILE,
    OPT_CHECKED, OPT_FP64_TRMM, OPT_FP64_TRSM, OPT_NVTX, OPT_RESIDUAL, OPT_SPLIT, OPT_THIN, OPT_THIN_LEAF, OPT_TRMM_DENSE, OPT_TRSM_DAG, OPT_TRSM_TC_LEAF, OPT_WAIT_LIMIT, RESIDUAL_AUTO, RESIDUAL_FLOAT_FLOAT,
    RESIDUAL_FP64, RESIDUAL_TC, Handle, TrxError, batched, batched_autotune, copy_triangle_h2d,
    debug_plan,
    default_handle,
    gemm_update, header_functions,
    load_library, load_tuning, peak_probe, save_tuning, to_colmajor, trmm, trsm, trsm_refined, trsm_refined_async,
)

__all__ = ["trsm", "trmm", "trsm_refined", "Handle", "TrxError", "default_handle", "debug_plan",
           "load_library", "to_colmajor"]
