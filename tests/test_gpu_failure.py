"""Failure detection without a fault: a bounded device wait that can never be
satisfied (an mbarrier nothing arrives at) gives up after its clock budget,
the kernel reports GSP_DEV_TIMEOUT through the status word, and the CUDA
context stays usable for the next launch."""
import time

import pytest
import torch

import synth
from _gpu import dev, lib, oracle_material, query_error, random_factors, QUERY_TOL

pytestmark = pytest.mark.gpu

GSP_DEV_TIMEOUT = 0x8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def test_bounded_wait_times_out_and_context_survives():
    import paper_2109_14807_gb300 as g
    torch.cuda.synchronize()
    t0 = time.time()
    st = g.selftest_wait_timeout()
    torch.cuda.synchronize()
    dt = time.time() - t0
    assert g.status_bits(st) & GSP_DEV_TIMEOUT
    assert 0.2 < dt < 30.0, dt  # the budget is about 2 s at GB300 clocks
    # the next launches run normally: a small query batch against the oracle
    f = random_factors(32, 6, 16, 16, 5)
    mat = g.QueryMaterial.from_factors({k: dev(v) for k, v in f.items()})
    g.build_query_tables(mat)
    q = synth.queries_fractional(32, 6, 16, 2000, 9)
    st2 = g.new_status()
    got = g.range_query(mat, g.queries_to_device(q), status=st2).cpu().numpy()
    assert g.status_bits(st2) == 0
    err, _ = query_error(got, oracle_material(f), q)
    assert err <= QUERY_TOL
