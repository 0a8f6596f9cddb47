"""GB300 (sm_103a) Self-Convolution block matching: C-ABI CUDA library + thin binding."""
from .bm import (BM_ALGO_AUTO, BM_ALGO_DIRECT, BM_ALGO_SELFCONV_TC, BM_F32, BM_OK, BM_U8,
                 BMError, Context, bm_aggregate, bm_check, bm_create, bm_destroy,
                 bm_gather_groups, bm_get_stats, bm_last_error, bm_match, bm_match_3d,
                 bm_match_batch, bm_match_direct, bm_match_host, bm_match_host_batch,
                 bm_match_ncc, bm_nlm, bm_num_refs, bm_poll, bm_request, bm_set_algo,
                 bm_set_fault_injection, bm_static_check, bm_static_init, bm_static_scratch_bytes,
                 bm_match_static, bm_submit, bm_window_split, bm_workspace_bytes, load)

__all__ = ["Context", "BMError", "load", "bm_create", "bm_destroy", "bm_last_error",
           "bm_num_refs", "bm_match", "bm_match_direct", "bm_match_host", "bm_match_batch",
           "bm_match_host_batch", "bm_set_algo", "bm_submit", "bm_poll", "bm_get_stats",
           "bm_request", "bm_check", "bm_set_fault_injection", "bm_gather_groups",
           "bm_aggregate", "bm_nlm", "bm_match_ncc", "bm_match_3d", "bm_match_static",
           "bm_static_scratch_bytes", "bm_static_init", "bm_static_check", "bm_window_split",
           "bm_workspace_bytes",
           "BM_U8", "BM_F32", "BM_OK", "BM_ALGO_AUTO", "BM_ALGO_DIRECT", "BM_ALGO_SELFCONV_TC"]
