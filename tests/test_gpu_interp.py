"""GPU parity of range queries at fractional texel positions (row f1, Sec. 4.1
interpolation between neighbouring footprints) against the FP64 oracle's
bilinear blend of integer-position queries."""
import numpy as np
import pytest
import torch

import synth
from oracle import query as oq
from _gpu import QUERY_TOL, lib, oracle_material, random_factors, to_device_factors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def _neighbour_kappa(mats, q):
    """Blend of the condition scales of the four neighbouring integer queries."""
    x0, y0 = np.floor(q["x"].astype(np.float64)), np.floor(q["y"].astype(np.float64))
    kap = np.zeros(len(q))
    for i in (0, 1):
        for j in (0, 1):
            qi = np.zeros(len(q), dtype=synth.QUERY_DTYPE)
            for k in ("level", "s0", "s1", "t0", "t1", "material"):
                qi[k] = q[k]
            qi["x"] = (x0 + i).astype(np.int64)
            qi["y"] = (y0 + j).astype(np.int64)
            w = np.where(i, q["x"] - x0, 1 - (q["x"] - x0)) * np.where(j, q["y"] - y0, 1 - (q["y"] - y0))
            kap += w * oq.condition_scale(mats, qi)
    return kap


@pytest.mark.parametrize("N,L,B,R", [(64, 7, 16, 16), (256, 9, 32, 64)])
def test_fractional_positions_match_oracle(N, L, B, R):
    import paper_2109_14807_gb300 as g
    f = random_factors(N, L, B, R, 600 + R)
    mat = g.QueryMaterial.from_factors(to_device_factors(f))
    g.build_query_tables(mat)
    om = oracle_material(f)
    q = synth.queries_fractional_xy(N, L, B, 50_000, 61)
    words = np.frombuffer(q.tobytes(), dtype=np.int32).reshape(-1, 8)
    st = g.new_status()
    got = g.range_query_interp(mat, torch.from_numpy(words.copy()).cuda(), status=st).cpu().numpy()
    assert g.status_bits(st) == 0
    ref = oq.cp_range_query_interp(om, q)
    kap = _neighbour_kappa(om, q)
    err = np.max(oq.kappa_relative_error(got.astype(np.float64), ref, kap))
    assert err <= QUERY_TOL, err


def test_integer_positions_equal_the_integer_query():
    import paper_2109_14807_gb300 as g
    f = random_factors(128, 8, 32, 32, 611)
    mat = g.QueryMaterial.from_factors(to_device_factors(f))
    g.build_query_tables(mat)
    qi = synth.queries_fractional(128, 8, 32, 20_000, 62, frac_level=True)
    qf = np.zeros(len(qi), dtype=synth.QUERY_F_DTYPE)
    for k in qi.dtype.names:
        qf[k] = qi[k]
    words = np.frombuffer(qf.tobytes(), dtype=np.int32).reshape(-1, 8)
    tn = (8, 8, 256, 4)
    a = g.range_query(mat, g.queries_to_device(qi), tuning=tn)
    b = g.range_query_interp(mat, torch.from_numpy(words.copy()).cuda(), tuning=tn)
    assert torch.equal(a, b)


def test_non_finite_position_is_a_bad_query():
    import paper_2109_14807_gb300 as g
    f = random_factors(32, 6, 16, 16, 612)
    mat = g.QueryMaterial.from_factors(to_device_factors(f))
    g.build_query_tables(mat)
    q = synth.queries_fractional_xy(32, 6, 16, 3, 63)
    q["x"][1] = np.inf
    q["y"][2] = 3e9
    words = np.frombuffer(q.tobytes(), dtype=np.int32).reshape(-1, 8)
    st = g.new_status()
    out = g.range_query_interp(mat, torch.from_numpy(words.copy()).cuda(), status=st).cpu().numpy()
    assert np.isfinite(out[0]) and np.isnan(out[1]) and np.isnan(out[2])
    assert g.status_bits(st) & 0x2
