"""GB300-native footprint-NDF binning, CP-ALS and constant-cost spatio-angular
range queries (Constant-Cost Spatio-Angular Prefiltering of Glinty Appearance
Using Tensor Decomposition, arXiv 2109.14807).

The compute lives in the CUDA library libgsp.so (C ABI: include/gsp.h); this
package is its Python binding.  Build it with ``paper_2109_14807_gb300.build.build()``.
"""
from .api import (CLUSTER_BLOCK, cluster_decompose, cluster_layout, cluster_range_query,
                  cluster_tables, CPWorkspace, QueryMaterial, RangeQueryFn, adam_step, backward_workspace_bytes,
                  bin_normals, env_queries, build_footprint_ndfs, build_query_tables, count_bins,
                  cp_decompose, init_factors_to_device, new_status, queries_to_device, range_query,
                  range_query_autograd, range_query_backward, range_query_interp, sample_ndf,
                  samples_to_device,
                  selftest_recip, selftest_wait_timeout, status_bits)

__all__ = [
    "CLUSTER_BLOCK", "cluster_decompose", "cluster_layout", "cluster_range_query", "cluster_tables",
    "CPWorkspace", "QueryMaterial", "RangeQueryFn", "adam_step", "backward_workspace_bytes",
    "bin_normals", "env_queries", "build_footprint_ndfs", "build_query_tables", "count_bins",
    "cp_decompose",
    "init_factors_to_device", "new_status", "queries_to_device", "range_query",
    "range_query_autograd", "range_query_backward", "range_query_interp", "sample_ndf",
    "samples_to_device",
    "selftest_recip", "selftest_wait_timeout", "status_bits",
]
