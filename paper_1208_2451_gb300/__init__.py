"""GB300 (sm_103a) LU_PRRP: blocked LU with panel rank revealing pivoting.

The compute path is libprrp.so (hand-written CUDA for sm_103a behind the C ABI in
include/prrp.h); this package is its Python binding.  Importing it fails loudly when the
library has not been built: there is no CPU fallback.
"""
from .binding import (KINDS, Server, partition_systems, prrp_batch_solve, prrp_server_create, PRRP_BF16X3, PRRP_FP32, PRRP_FP64, PRRP_TF32, STATUS, Context,
                      Factors, PrrpError, default_opts, exported_symbols, prrp_create,
                      prrp_ctx_kernel_stats, prrp_ctx_set_panel_mode, prrp_ctx_set_sm_split, prrp_ctx_set_update_block, prrp_ctx_set_timing, prrp_factor_calu, prrp_factor_block, prrp_ctx_timeline, prrp_destroy,
                      prrp_factor, prrp_gesv_host, prrp_panel_select, prrp_panel_select_noalloc,
                      prrp_schur_update, prrp_selftest_wait, prrp_selftest_chain_wait, prrp_ctx_set_solve_mode, prrp_batch_tune,
                      prrp_solve, prrp_status_string, prrp_version)

__all__ = ["KINDS", "Server", "partition_systems", "prrp_batch_solve", "prrp_server_create", "PRRP_BF16X3", "PRRP_FP32", "PRRP_FP64", "PRRP_TF32", "STATUS", "Context",
           "Factors", "PrrpError", "default_opts", "exported_symbols", "prrp_create",
           "prrp_ctx_kernel_stats", "prrp_ctx_set_panel_mode", "prrp_ctx_set_sm_split", "prrp_ctx_set_update_block", "prrp_ctx_set_timing", "prrp_factor_calu", "prrp_factor_block", "prrp_ctx_timeline", "prrp_destroy", "prrp_factor",
           "prrp_gesv_host", "prrp_panel_select", "prrp_panel_select_noalloc", "prrp_schur_update", "prrp_selftest_wait", "prrp_selftest_chain_wait", "prrp_ctx_set_solve_mode", "prrp_batch_tune",
           "prrp_solve", "prrp_status_string", "prrp_version"]
