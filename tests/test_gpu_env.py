"""GPU parity of the environment-prefiltering query generator (row f4, Sec.
5.4) against the FP64 oracle, and of the range queries it feeds."""
import numpy as np
import pytest
import torch

import synth
from oracle import query as oq
from _gpu import QUERY_TOL, lib, oracle_material, random_factors, to_device_factors

pytestmark = pytest.mark.gpu

SHAPES = [(128, 16, 16), (256, 32, 32), (512, 64, 64)]  # (N, rank, bins)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def _words(a):
    return torch.from_numpy(np.frombuffer(np.ascontiguousarray(a).tobytes(), dtype=np.int32)
                            .reshape(len(a), -1).copy()).cuda()


def test_env_queries_match_oracle_and_feed_range_queries():
    import paper_2109_14807_gb300 as g
    mats, omats, dims = [], [], []
    for i, (N, R, B) in enumerate(SHAPES):
        L = int(np.log2(N)) + 1
        f = random_factors(N, L, B, R, 700 + i)
        m = g.QueryMaterial.from_factors(to_device_factors(f))
        g.build_query_tables(m)
        mats.append(m)
        omats.append(oracle_material(f))
        dims.append((N, L, B))
    sgs = synth.env_lobes(24, 71)
    rec = synth.env_records(dims, 100_000, len(sgs), 72)
    sg_t = torch.from_numpy(sgs.view(np.float32).reshape(len(sgs), 8).copy()).cuda()
    qd = g.env_queries(mats, sg_t, _words(rec))
    qg = np.frombuffer(qd.cpu().numpy().tobytes(), dtype=synth.QUERY_DTYPE)
    ref = oq.env_queries(sgs, rec, [d[2] for d in dims])
    assert np.array_equal(qg["x"], ref["x"]) and np.array_equal(qg["y"], ref["y"])
    assert np.array_equal(qg["material"], ref["material"]) and np.array_equal(qg["level"], rec["level"])
    for k in ("s0", "s1", "t0", "t1"):  # bins; FP32 transcendental and normalisation rounding
        assert np.max(np.abs(qg[k] - ref[k])) <= 2e-4 * 64, k
    st = g.new_status()
    out = g.range_query(mats, qd, status=st).cpu().numpy().astype(np.float64)
    assert g.status_bits(st) == 0
    refq = oq.cp_range_query(omats, qg)
    kap = oq.condition_scale(omats, qg)
    assert np.max(oq.kappa_relative_error(out, refq, kap)) <= QUERY_TOL


def test_bad_records_make_bad_queries():
    import paper_2109_14807_gb300 as g
    N, R, B = 64, 16, 16
    f = random_factors(N, 7, B, R, 710)
    m = g.QueryMaterial.from_factors(to_device_factors(f))
    g.build_query_tables(m)
    sgs = synth.env_lobes(2, 73)
    rec = synth.env_records([(N, 7, B)], 3, 2, 74)
    rec["sg"][1] = 9                      # no such lobe
    rec["wo"][2] = -sgs["axis"][rec["sg"][2]]  # wo = -axis: no half vector
    sg_t = torch.from_numpy(sgs.view(np.float32).reshape(len(sgs), 8).copy()).cuda()
    qd = g.env_queries([m], sg_t, _words(rec))
    st = g.new_status()
    out = g.range_query([m], qd, status=st).cpu().numpy()
    assert np.isfinite(out[0]) and np.isnan(out[1]) and np.isnan(out[2])
    assert g.status_bits(st) & 0x2
