"""Exact, deterministic 1-NN search over Hierarchical-Normalization descriptors on B300 (sm_103a).

The compute lives in libhn.so (CUDA, C ABI in include/hn.h); ``hn`` is its
ctypes binding.  Importing this package loads the library and raises
ImportError if it has not been built.
"""
from .hn import (D, HNError, Index, PREFIX_BF16, merge_topk, merge_topk_host, PREFIX_F32, PREFIX_FP8, PREFIX_I8, Proposal, RESCORE_BEST_FIRST, RESCORE_FILTER16, RESCORE_FULL, SCAN_AUTO, SCAN_DENSE,
                 SCAN_DENSE_TWO_PASS, SCAN_STREAM,
                 SearchResult, gemm_bf16, linear_bf16, mlp_loss_grad, normalize, normalize_async, search_multi, selftest_wait_timeout, version)

__all__ = ["D", "HNError", "Index", "PREFIX_BF16", "merge_topk", "merge_topk_host", "PREFIX_F32", "PREFIX_FP8", "PREFIX_I8", "Proposal", "RESCORE_BEST_FIRST", "RESCORE_FILTER16", "RESCORE_FULL",
           "SCAN_AUTO", "SCAN_DENSE",
           "SCAN_DENSE_TWO_PASS", "SCAN_STREAM", "SearchResult", "gemm_bf16", "linear_bf16", "mlp_loss_grad", "normalize", "normalize_async",
           "search_multi", "selftest_wait_timeout",
           "version"]
