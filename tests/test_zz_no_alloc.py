"""The no-allocation variant of the range-query adjoint.

Some callers cannot allocate device memory -- a shading plugin that only gets
the device pointers its host renderer hands it, or a frame loop that must not
call cudaMalloc because it synchronises the device.  For them the library
offers gsp_range_query_backward_noalloc, which takes its scratch from a fixed
array inside the library instead of a caller workspace.  This test calls it
through the C ABI twice in a row and checks both results against the
workspace version, within the adjoint tolerance of the other GPU tests.  It
lives in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import query as oq
from _gpu import dev, lib, oracle_material, random_factors

pytestmark = pytest.mark.gpu
NAMES = (("dfx", "fx"), ("dfy", "fy"), ("dflw", "flw"), ("dfs", "fs"), ("dft", "ft"))


def _zero_grads(f):
    return {k: torch.zeros(f[a if a != "flw" else "fl"].shape, dtype=torch.float32, device="cuda")
            for k, a in NAMES}


def test_backward_noalloc_matches_workspace_version():
    import paper_2109_14807_gb300 as g
    from paper_2109_14807_gb300 import _lib
    L_ = lib()
    shapes = [(32, 6, 16, 16), (64, 7, 32, 64)]
    fs = [random_factors(N, L, B, R, 90 + i) for i, (N, L, B, R) in enumerate(shapes)]
    mats = []
    for f in fs:
        m = g.QueryMaterial.from_factors({k: dev(v) for k, v in f.items()})
        g.build_query_tables(m)
        mats.append(m)
    q = np.concatenate([
        synth.queries_fractional(32, 6, 16, 3000, 91, wmin=0.05, wmax=16, frac_level=True),
        synth.queries_fractional(64, 7, 32, 3000, 92, wmin=0.05, wmax=32, frac_level=True, material=1)])
    q[7]["s1"] = q[7]["s0"]
    q[3001]["t0"] = q[3001]["t1"]
    qd = g.queries_to_device(q)
    gup = (synth.uniform(93, 1, len(q)) - 0.5).astype(np.float32)
    gd = dev(gup)

    ref = [_zero_grads(f) for f in fs]
    g.range_query_backward(mats, qd, gd, ref)

    arr = (_lib.Material * len(mats))(*[m.struct() for m in mats])
    stream = torch.cuda.current_stream().cuda_stream
    status = g.new_status()
    om = [oracle_material(f) for f in fs]
    scale = oq.cp_range_query_adjoint([{k: np.abs(v) for k, v in o.items()} for o in om], q,
                                      np.abs(gup.astype(np.float64)))
    for call in range(2):
        got = [_zero_grads(f) for f in fs]
        garr = (_lib.MaterialGrad * len(mats))(*[
            _lib.MaterialGrad(*(gr[k].data_ptr() for k, _ in NAMES)) for gr in got])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = L_.gsp_range_query_backward_noalloc(arr, len(mats), qd.data_ptr(), qd.shape[0],
                                                 gd.data_ptr(), garr, status.data_ptr(), stream)
        assert rc == 0, rc
        torch.cuda.synchronize()
        if call == 1:
            # the device's free memory is the same after the call: the library
            # took no device memory of its own (the first call may have loaded
            # the module, whose globals hold the scratch array)
            assert torch.cuda.mem_get_info()[0] == free0
        assert g.status_bits(status) == 0
        for mi in range(len(mats)):
            for k, a in NAMES:
                diff = (got[mi][k] - ref[mi][k]).abs().double().cpu().numpy()
                err = np.max(diff / np.maximum(scale[mi][a], 1e-30))
                assert err <= 1e-4, (call, mi, k, err)


def test_backward_noalloc_rejects_oversized_scratch():
    from paper_2109_14807_gb300 import _lib
    L_ = lib()
    # 16 materials of B = 128, R = 256 need 16 * 2 * 129 * 256 * 4 bytes > 4 MiB
    m = _lib.Material(1024, 11, 128, 256, 1, 1, 1, 1, 1, 1, 256)
    arr = (_lib.Material * 16)(*([m] * 16))
    gr = _lib.MaterialGrad(1, 1, 1, 1, 1)
    garr = (_lib.MaterialGrad * 16)(*([gr] * 16))
    assert L_.gsp_backward_workspace_bytes(arr, 16) > (4 << 20)
    rc = L_.gsp_range_query_backward_noalloc(arr, 16, None, 0, None, garr, None, None)
    assert rc == -3  # GSP_ERR_WORKSPACE, nothing enqueued
    # a malformed material (map side not a power of two) is an argument error,
    # even where the scratch it asks for is also too large
    bad = _lib.Material(1000, 11, 128, 256, 1, 1, 1, 1, 1, 1, 256)
    arr_bad = (_lib.Material * 16)(*([bad] * 16))
    assert L_.gsp_range_query_backward_noalloc(arr_bad, 16, None, 0, None, garr, None, None) == -1
