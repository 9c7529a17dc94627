"""ctypes declarations of the C ABI in include/gsp.h (argument marshalling only).

The shared library is loaded lazily on first use.  If it has not been built the
call fails loudly: there is no CPU fallback for any operation.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import (POINTER, Structure, c_char_p, c_double, c_float, c_int, c_int32, c_int64,
                    c_size_t, c_uint32, c_void_p)

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgsp.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "gsp.h")

GSP_OK = 0
STATUS_NAMES = {0: "GSP_OK", -1: "GSP_ERR_INVALID_ARG", -2: "GSP_ERR_CUDA", -3: "GSP_ERR_WORKSPACE",
                -4: "GSP_ERR_NONFINITE", -5: "GSP_ERR_NUMERIC", -6: "GSP_ERR_TIMEOUT",
                -7: "GSP_ERR_UNSUPPORTED"}
DEV_NONFINITE_NORMAL = 0x1
DEV_BAD_QUERY = 0x2
DEV_NUMERIC = 0x4
DEV_TIMEOUT = 0x8
MAX_MATERIALS = 16
MAX_SWEEPS = 512
PREC = {"fp32": 0, "tf32": 1, "bf16": 2, "bf16_1x": 3, "structured": 4,
        "structured_gaussian": 5}


class Material(Structure):
    _fields_ = [("N", c_int32), ("levels", c_int32), ("bins", c_int32), ("rank", c_int32),
                ("fx", c_void_p), ("fy", c_void_p), ("fl", c_void_p), ("fs", c_void_p),
                ("ft", c_void_p), ("lam", c_void_p), ("tables", c_void_p)]


class MaterialGrad(Structure):
    _fields_ = [("dfx", c_void_p), ("dfy", c_void_p), ("dflw", c_void_p), ("dfs", c_void_p),
                ("dft", c_void_p)]


class CpFactors(Structure):
    _fields_ = [("fx", c_void_p), ("fy", c_void_p), ("fl", c_void_p), ("fs", c_void_p),
                ("ft", c_void_p), ("lam", c_void_p)]


class AlsOpts(Structure):
    _fields_ = [("sweeps", c_int32), ("precision", c_int32), ("tol", c_double),
                ("raw_counts", c_int32), ("reserved", c_int32)]


class AlsReport(Structure):
    _fields_ = [("sweeps_done", c_int32), ("numeric_fallbacks", c_int32),
                ("fit", c_double * MAX_SWEEPS)]


class QueryTuning(Structure):
    _fields_ = [("lanes_per_query", c_int32), ("blocks_per_sm", c_int32), ("threads", c_int32),
                ("chunk", c_int32)]


_SIGS = {
    "gsp_bin_normals": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "gsp_build_workspace_bytes": (c_size_t, [c_int, c_int, c_int]),
    "gsp_build_footprint_ndfs": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p,
                                         c_size_t, c_void_p, c_void_p]),
    "gsp_cp_workspace_bytes": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "gsp_cp_workspace_bytes_for_bins": (c_size_t, [c_int, c_int, c_int, c_int, c_int, c_int]),
    "gsp_cp_count_bins_workspace_bytes": (c_size_t, [c_int, c_int]),
    "gsp_cp_count_bins": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_size_t,
                                  POINTER(c_int32), c_void_p, c_void_p]),
    "gsp_cp_operand_offset": (c_size_t, [c_int, c_int, c_int, c_int, c_int]),
    "gsp_cp_prepare": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, POINTER(AlsOpts),
                               c_void_p, c_size_t, c_void_p, c_void_p]),
    "gsp_cp_sweeps": (c_int, [c_int, c_int, c_int, c_int, POINTER(AlsOpts), POINTER(CpFactors),
                              POINTER(AlsReport), c_void_p, c_size_t, c_void_p]),
    "gsp_cp_decompose": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, POINTER(AlsOpts),
                                 POINTER(CpFactors), POINTER(AlsReport), c_void_p, c_size_t,
                                 c_void_p, c_void_p]),
    "gsp_cp_mttkrp": (c_int, [c_int, c_int, c_int, c_int, c_int, POINTER(CpFactors),
                              POINTER(c_void_p), c_void_p, c_size_t, c_void_p]),
    "gsp_query_table_floats": (c_size_t, [c_int, c_int, c_int]),
    "gsp_build_query_tables": (c_int, [POINTER(Material), c_void_p]),
    "gsp_range_query": (c_int, [POINTER(Material), c_int, c_void_p, c_int64, c_void_p, c_void_p,
                                POINTER(QueryTuning), c_void_p, c_size_t, c_void_p]),
    "gsp_sample_ndf": (c_int, [POINTER(Material), c_int, c_void_p, c_int64, c_void_p, c_void_p,
                               c_void_p, c_void_p]),
    "gsp_cp_operand_cols": (c_int, [c_int, c_int, c_int, c_int, c_int, c_void_p, c_size_t,
                                    POINTER(c_int32), c_void_p]),
    "gsp_cluster_groups": (c_int, [c_int, c_int, c_int]),
    "gsp_cluster_layout_bytes": (c_size_t, [c_int, c_int, c_int]),
    "gsp_cluster_layout": (c_int, [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                   POINTER(c_int64), c_void_p, c_size_t, c_void_p]),
    "gsp_cluster_als_smem": (c_size_t, [c_int, c_int]),
    "gsp_cluster_als": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_int,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_double, c_int,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gsp_cluster_tables": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "gsp_cluster_range_query": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p,
                                        c_void_p]),
    "gsp_env_queries": (c_int, [POINTER(Material), c_int, c_void_p, c_int, c_void_p, c_int64,
                                c_float, c_void_p, c_void_p]),
    "gsp_range_query_interp": (c_int, [POINTER(Material), c_int, c_void_p, c_int64, c_void_p,
                                       c_void_p, POINTER(QueryTuning), c_void_p, c_size_t,
                                       c_void_p]),
    "gsp_backward_workspace_bytes": (c_size_t, [POINTER(Material), c_int]),
    "gsp_range_query_backward": (c_int, [POINTER(Material), c_int, c_void_p, c_int64, c_void_p,
                                         POINTER(MaterialGrad), c_void_p, c_size_t, c_void_p,
                                         c_void_p]),
    "gsp_range_query_backward_noalloc": (c_int, [POINTER(Material), c_int, c_void_p, c_int64,
                                                 c_void_p, POINTER(MaterialGrad), c_void_p,
                                                 c_void_p]),
    "gsp_adam_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int, c_float,
                              c_float, c_float, c_float, c_void_p]),
    "gsp_profile_enable": (c_int, [c_int]),
    "gsp_profile_reset": (None, []),
    "gsp_profile_read": (c_int, [c_int, POINTER(c_int64), POINTER(c_double)]),
    "gsp_profile_name": (c_char_p, [c_int]),
    "gsp_kernel_launches": (ctypes.c_uint64, []),
    "gsp_strerror": (c_char_p, [c_int]),
    "gsp_last_cuda_error": (c_int, []),
    "gsp_version": (c_int, []),
    "gsp_selftest_wait_timeout": (c_int, [c_void_p, c_void_p]),
    "gsp_selftest_recip": (c_int, [c_void_p, c_int64, c_void_p, c_void_p]),
}

_LIB = None


def header_symbols() -> list:
    """Every function name declared in include/gsp.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsp_[a-z0-9_]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load the library (once) and declare every entry point's signature."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is not built; run paper_2109_14807_gb300.build.build() first "
            "(every operation runs in the CUDA library; there is no fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class GspError(RuntimeError):
    def __init__(self, fn: str, code: int):
        lib = _LIB
        msg = lib.gsp_strerror(code).decode() if lib is not None else STATUS_NAMES.get(code, "?")
        extra = ""
        if code == -2 and lib is not None:
            extra = f" (cudaError {lib.gsp_last_cuda_error()})"
        super().__init__(f"{fn} failed: {STATUS_NAMES.get(code, code)}: {msg}{extra}")
        self.code = code


def check(fn: str, code: int) -> None:
    if code != GSP_OK:
        raise GspError(fn, code)
