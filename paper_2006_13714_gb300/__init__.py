"""GB300 (sm_103a) Self-Convolution block matching: C-ABI CUDA library + thin binding."""
from .bm import (BM_ALGO_AUTO, BM_ALGO_DIRECT, BM_ALGO_SELFCONV_TC, BM_F32, BM_OK, BM_U8,
                 BMError, Context, bm_create, bm_destroy, bm_get_stats, bm_last_error,
                 bm_match, bm_match_batch, bm_match_direct, bm_match_host, bm_num_refs,
                 bm_poll, bm_request, bm_set_algo, bm_submit, load)

__all__ = ["Context", "BMError", "load", "bm_create", "bm_destroy", "bm_last_error",
           "bm_num_refs", "bm_match", "bm_match_direct", "bm_match_host", "bm_match_batch",
           "bm_set_algo", "bm_submit", "bm_poll", "bm_get_stats", "bm_request",
           "BM_U8", "BM_F32", "BM_OK", "BM_ALGO_AUTO", "BM_ALGO_DIRECT", "BM_ALGO_SELFCONV_TC"]
