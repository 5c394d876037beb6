"""GB300-native compressed matrix multiplication (Pagh, arXiv 1108.1320).

The compute path is libcms.so (hand-written sm_103a CUDA kernels behind the C
ABI of include/cms.h); ``paper_1108_1320_gb300.cms`` is its Python binding.
"""
from .cms import (KERNEL_NAMES, Batch, CmsError, Hashes, alloc_workspace, check_async, decode, decode_dense,
                  decode_significant, decode_threshold, find_significant, frobenius_estimate, lib, make_hashes,
                  merge, nnz_estimate, plain_workspace_size, plan_kernel, profile_enable, profile_summary,
                  remove_diagonal, selftest_wait, sketch_product, sketch_product_csr, sketch_product_noalloc,
                  sketch_product_plain_f64, sparse_workspace_size, status_string, workspace_size)

__all__ = ["KERNEL_NAMES", "Batch", "CmsError", "Hashes", "alloc_workspace", "check_async", "decode", "decode_dense",
           "decode_significant", "decode_threshold", "find_significant", "frobenius_estimate", "lib",
           "make_hashes", "merge", "nnz_estimate", "plain_workspace_size", "plan_kernel", "profile_enable",
           "profile_summary", "remove_diagonal", "selftest_wait", "sketch_product", "sketch_product_csr", "sketch_product_noalloc",
           "sketch_product_plain_f64", "sparse_workspace_size", "status_string", "workspace_size"]
