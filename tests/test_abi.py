"""The C-ABI library builds for sm_103a, loads, and exports every symbol
include/gsp.h declares; host-side argument checks answer without a GPU."""
import ctypes
import shutil

import pytest

from paper_2109_14807_gb300 import _lib, build

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not build.up_to_date(),
                                reason="nvcc not available to build libgsp.so")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _lib.header_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every declared function has a ctypes signature in the binding
    assert set(names) == set(_lib._SIGS)


def test_struct_sizes_match_header():
    assert ctypes.sizeof(_lib.Material) == 16 + 7 * 8
    assert ctypes.sizeof(_lib.AlsOpts) == 24
    assert ctypes.sizeof(_lib.AlsReport) == 8 + 8 * _lib.MAX_SWEEPS
    assert ctypes.sizeof(_lib.QueryTuning) == 16
    assert ctypes.sizeof(_lib.CpFactors) == 6 * 8
    import synth
    assert synth.QUERY_DTYPE.itemsize == 32


def test_host_side_sizes_and_validation(lib):
    assert lib.gsp_version() >= 10000
    assert lib.gsp_strerror(0) == b"ok"
    assert lib.gsp_strerror(-3) == b"workspace too small"
    # sizes
    assert lib.gsp_build_workspace_bytes(32, 6, 16) >= 32 * 32 * 2
    assert lib.gsp_build_workspace_bytes(33, 6, 16) == 0          # N not a power of two
    assert lib.gsp_build_workspace_bytes(32, 7, 16) == 0          # too many levels
    assert lib.gsp_query_table_floats(6, 16, 8) == 6 * 8 + 6 * 17 * 8
    assert lib.gsp_query_table_floats(5, 8, 3) == 16 + 6 * 9 * 3   # flw padded to 4 floats
    assert lib.gsp_cp_workspace_bytes(32, 6, 16, 8, 0) > 32 * 32 * 6 * 256 * 4
    assert lib.gsp_cp_workspace_bytes(32, 6, 16, 12, 0) == 0      # rank not a power of two
    assert lib.gsp_cp_workspace_bytes(32, 6, 16, 8, 3) == 0       # unknown precision
    # workspace sized by the occupied bins: all bins give the worst case, fewer
    # a smaller one with the same head (operand offset).  The FP32 path stores
    # the occupied bins rounded up to 128 columns: 67 bins of the 1024^2 / 11
    # levels / 32^2 bins / rank 64 shape take 128 columns (5.9 GB of operand)
    # instead of 1024 (47 GB).  (The tensor-core precisions need the driver's
    # tensor-map encoder, absent without a GPU: their sizes are tested on one.)
    fp32 = _lib.PREC["fp32"]
    full = lib.gsp_cp_workspace_bytes(1024, 11, 32, 64, fp32)
    assert lib.gsp_cp_workspace_bytes_for_bins(1024, 11, 32, 64, fp32, 1024) <= full
    occ = lib.gsp_cp_workspace_bytes_for_bins(1024, 11, 32, 64, fp32, 67)
    assert 1024 * 1024 * 11 * 128 * 4 < occ < 7 << 30 < full
    assert lib.gsp_cp_workspace_bytes_for_bins(1024, 11, 32, 64, fp32, 0) == 0
    assert lib.gsp_cp_workspace_bytes_for_bins(1024, 11, 32, 64, fp32, 1025) == 0
    sizes = [lib.gsp_cp_workspace_bytes_for_bins(128, 8, 32, 16, fp32, n) for n in (1, 100, 300, 1024)]
    assert sizes == sorted(sizes) and sizes[-1] <= lib.gsp_cp_workspace_bytes(128, 8, 32, 16, fp32)
    assert sizes[0] == sizes[1] and sizes[1] < sizes[2]  # 1 and 100 bins: both 128 columns
    off = lib.gsp_cp_operand_offset(1024, 11, 32, 64, fp32)
    assert off >= 1024 * 1024 * 2 and off % 256 == 0
    assert lib.gsp_cp_operand_offset(1024, 11, 32, 64, _lib.PREC["structured"]) == 0
    assert lib.gsp_cp_count_bins_workspace_bytes(1024, 32) >= 1024 * 1024 * 2
    assert lib.gsp_cp_count_bins(None, None, 32, 6, 16, None, 0, None, None, None) == -1
    # argument errors are returned before anything is enqueued
    assert lib.gsp_build_footprint_ndfs(None, 32, 6, 16, None, None, 0, None, None) == -1
    # a NULL histogram is the implicit form: accepted, so a missing workspace is the error
    fake = ctypes.c_void_p(4096)
    assert lib.gsp_build_footprint_ndfs(fake, 32, 6, 16, None, None, 0, None, None) == -3
    assert lib.gsp_build_footprint_ndfs(fake, 32, 6, 16, None, fake, 2047, None, None) == -3
    assert lib.gsp_build_footprint_ndfs(fake, 33, 6, 16, None, fake, 1 << 20, None, None) == -1
    assert lib.gsp_range_query(None, 1, None, 10, None, None, None, None, 0, None) == -1
    m = _lib.Material()
    assert lib.gsp_range_query(ctypes.byref(m), 0, None, 0, None, None, None, None, 0, None) == -1
    assert lib.gsp_range_query(ctypes.byref(m), 17, None, 0, None, None, None, None, 0, None) == -1
    assert lib.gsp_adam_step(None, None, None, None, 5, 1, 1e-3, 0.9, 0.999, 1e-8, None) == -1
    opts = _lib.AlsOpts(0, 0, 0.0, 0, 0)
    f = _lib.CpFactors()
    assert lib.gsp_cp_sweeps(32, 6, 16, 8, ctypes.byref(opts), ctypes.byref(f), None, None, 0,
                             None) == -1


def test_backward_workspace_holds_the_private_copies(lib):
    # the adjoint's scratch: each material's summed-area-table prefix-row
    # gradients (2 (B+1) R floats, 256-byte aligned each), then 128 private
    # copies of every material's small gradient tables ((L + 2 (B+1)) R floats)
    def align(b):
        return -(-b // 256) * 256

    shapes = [(1024, 11, 32, 64), (64, 7, 32, 64), (32, 6, 16, 16)]
    mats = [_lib.Material(N, L, B, R, 1, 1, 1, 1, 1, 1, 1) for N, L, B, R in shapes]
    arr = (_lib.Material * len(mats))(*mats)
    want = sum(2 * align((B + 1) * R * 4) for _, _, B, R in shapes)
    want += align(128 * sum((L + 2 * (B + 1)) * R for _, L, B, R in shapes) * 4)
    assert lib.gsp_backward_workspace_bytes(arr, len(mats)) == want
    # one material of the 1024^2 / 11-level / 32^2-bin / rank-64 shape fits the
    # no-allocation entry's fixed array
    assert lib.gsp_backward_workspace_bytes(arr, 1) <= 4 << 20
    assert lib.gsp_backward_workspace_bytes(arr, 0) == 0
