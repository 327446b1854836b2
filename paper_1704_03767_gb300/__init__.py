"""GB300-native exact all-pairs Kendall tau-b (Liu et al., arXiv 1704.03767).

The computation lives in libktau.so (hand-written sm_103a CUDA behind the C ABI in
include/ktau.h); this package is its thin ctypes binding. Build the library with
``python -m paper_1704_03767_gb300.build``.
"""
from .binding import (  # noqa: F401
    KTAU_F32,
    KTAU_I32,
    KTAU_MAX_N,
    KTAU_PATH_AUTO,
    KTAU_PATH_MERGE,
    KTAU_PATH_SIGNGEMM,
    Batch,
    BatchDesc,
    KtauError,
    Options,
    Ranked,
    allpairs,
    batch_desc,
    declared_symbols,
    ktau_allpairs,
    ktau_allpairs_host,
    ktau_allpairs_noalloc,
    ktau_allpairs_path,
    ktau_debug_fail_alloc,
    ktau_permutation_exceed,
    permutation_pvalues,
    ktau_debug_wait_timeout,
    ktau_device_status,
    ktau_prepare_signs,
    ktau_query,
    ktau_query_scratch_bytes,
    ktau_rank_prepare,
    ktau_rank_prepare_async,
    ktau_ranked_export,
    ktau_tie_counts,
    ktau_trace_collect,
    ktau_trace_enable,
    ktau_trace_filter,
    load,
)
