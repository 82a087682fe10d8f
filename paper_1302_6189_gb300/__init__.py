"""GB300-native (sm_103a) M-D complex FFT with the row-wise adaptive
decomposition and transpose-order awareness of Duy and Ozaki
(arXiv:1302.6189).  The compute path is libmdfft (include/mdfft.h); this
package is its thin binding."""

from .mdfft import (  # noqa: F401
    DTYPES, MDFFT_C64, MDFFT_C128, MDFFT_C64_TC_BF16, MDFFT_C64_TC_FP16, MDFFT_PLAN_HOST_ONLY,
    MDFFT_PLAN_INPLACE, MDFFT_PLAN_PERSISTENT, MDFFT_PLAN_DECOMP_SLAB, MDFFT_PLAN_DECOMP_PENCIL, MDFFT_PLAN_OUT_NATURAL, MDFFT_PLAN_OUT_LAST_LAYOUT, MDFFT_PLAN_TUNE_RADIX,
    MDFFT_PLAN_DECOMP_VOLUMETRIC, DECOMPOSITIONS, LIB_PATH, MdfftError, Plan, Server, format_order, mdfft_chunk, mdfft_comm_volume,
    mdfft_destroy, mdfft_exec, mdfft_exec_counted, mdfft_exec_graph, mdfft_selftest_wait, mdfft_exec_host, mdfft_exec_noalloc, mdfft_exchange_counts, mdfft_block_grid, mdfft_last_error, mdfft_launches_per_exec,
    mdfft_order_heuristic, mdfft_order_search, mdfft_pass_describe, mdfft_pass_times, mdfft_pass_timing, mdfft_plan, mdfft_plan_batched, mdfft_plan_tuning, mdfft_plan_set_tuning,
    mdfft_plan_order, mdfft_supported_length, mdfft_workspace_size, mdfft_fp64_rate_probe, parse_order,
    DistPlan, torch_exchange, mdfft_dist_local_range, mdfft_dist_lines, mdfft_dist_pack, mdfft_dist_unpack)
