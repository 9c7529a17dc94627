"""GPU parity of the query tables and batched range queries (rows a5-a6)
against the FP64 oracle on the same factors: kappa-relative error <= 1e-5."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import query as oq
from _gpu import QUERY_TOL, dev, lib, oracle_material, query_error, random_factors, \
    to_device_factors

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def _material(f):
    import paper_2109_14807_gb300 as g
    m = g.QueryMaterial.from_factors(to_device_factors(f))
    g.build_query_tables(m)
    return m


def _run(mats, q, **kw):
    import paper_2109_14807_gb300 as g
    st = g.new_status()
    out = g.range_query(mats, g.queries_to_device(q), status=st, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy(), g.status_bits(st)


def test_tables_layout():
    f = random_factors(8, 4, 8, 5, 1)
    m = _material(f)
    tab = m.tables.cpu().numpy()
    L, B, R = 4, 8, 5
    flw = tab[:L * R].reshape(L, R)
    assert np.allclose(flw, f["fl"] * f["lambda"][None], rtol=1e-7, atol=0)
    assert tab.size == (L * R + 3) // 4 * 4 + 2 * (B + 1) * 3 * R
    sat = tab[(L * R + 3) // 4 * 4:].reshape(2, B + 1, 3, R)  # [side][i][hi, lo, f][r]
    for side, fk in ((0, "fs"), (1, "ft")):
        P = oq.prefix_table(f[fk].astype(np.float64))
        hi, lo = sat[side, :, 0].astype(np.float64), sat[side, :, 1].astype(np.float64)
        assert np.all(np.abs(hi + lo - P) <= 1e-14 * np.maximum(1, np.abs(P)))
        assert np.array_equal(sat[side, :B, 2], f[fk])
        assert np.all(sat[side, B, 2] == 0)


def test_golden_rank2_hand_worked():
    f = dict(fx=np.array([[1, 1], [3, -1]], np.float32), fy=np.array([[2, 1], [1, 1]], np.float32),
             fl=np.array([[0.5, 1], [1.5, 2]], np.float32),
             fs=np.array([[1, 0], [2, 1], [3, 0], [4, 1]], np.float32),
             ft=np.array([[4, 1], [0, 1], [2, 1], [2, 1]], np.float32),
             **{"lambda": np.ones(2, np.float32)})
    rows = np.loadtxt(os.path.join(GOLDEN, "range_query_rank2.txt"), comments="#")
    q = np.zeros(len(rows), dtype=synth.QUERY_DTYPE)
    for i, r in enumerate(rows):
        q[i] = (int(r[0]), int(r[1]), r[2], r[3], r[4], r[5], r[6], 0)
    got, st = _run(_material(f), q)
    assert st == 0
    assert np.allclose(got, rows[:, 7], rtol=1e-6, atol=0)


@pytest.mark.parametrize("R,lanes", [(8, None), (8, 4), (8, 32), (37, None), (64, None), (64, 16)])
def test_integer_queries_tiny_shape(R, lanes):
    f = random_factors(32, 6, 16, R, 100 + R)
    q = synth.queries_integer(32, 6, 16, 10_000, 1001)
    tuning = None if lanes is None else (lanes, 4, 256, 2)
    got, st = _run(_material(f), q, tuning=tuning)
    assert st == 0
    err, _ = query_error(got, oracle_material(f), q)
    assert err <= QUERY_TOL


def test_fractional_queries_fractional_levels():
    f = random_factors(64, 7, 32, 32, 7)
    q = synth.queries_fractional(64, 7, 32, 50_000, 8, wmin=0.01, wmax=32, frac_level=True)
    got, st = _run(_material(f), q)
    assert st == 0
    err, _ = query_error(got, oracle_material(f), q)
    assert err <= QUERY_TOL


def test_ranges_ending_in_blank_bins():
    # a CP material whose angular factors are large in some bins and exactly 0
    # in others (blank regions of the NDF images): ranges that start just
    # before the end of a large bin and run into zeros have a tiny integral;
    # it must not be the difference of two large prefix sums
    f = random_factors(32, 6, 32, 16, 17, signed=True)
    for k in ("fs", "ft"):
        f[k][6:20] = 0.0
        f[k][5] *= 40.0
        f[k][20] *= 40.0
    u = synth.uniform(91, 1, 5 * 4000).reshape(4000, 5)
    q = np.zeros(4000, dtype=synth.QUERY_DTYPE)
    q["x"] = (u[:, 0] * 32).astype(np.int32)
    q["y"] = (u[:, 1] * 32).astype(np.int32)
    q["level"] = (u[:, 2] * 5).astype(np.float32)
    q["s0"] = (6.0 - 10.0 ** (-1.0 - 4.0 * u[:, 3])).astype(np.float32)  # just before 6
    q["s1"] = (6.0 + 13.0 * u[:, 4]).astype(np.float32)
    q["t0"] = (20.0 - 14.0 * u[:, 3]).astype(np.float32)
    q["t1"] = (20.0 + 10.0 ** (-1.0 - 4.0 * u[:, 4])).astype(np.float32)  # just past 20
    got, st = _run(_material(f), q)
    assert st == 0
    err, _ = query_error(got, oracle_material(f), q)
    assert err <= QUERY_TOL, err


def test_scale_shape_ten_million_queries_sampled():
    # 1024^2 map, 11 levels, 32 bins, rank 64; 10^7 fractional queries in the
    # launch configuration the benchmark times; every output finite, a sample
    # of 200k checked against the oracle
    w = synth.WORKLOADS["flakes1024"]
    f = random_factors(w["N"], w["levels"], w["bins"], w["rank"], 3)
    q = synth.queries_fractional(w["N"], w["levels"], w["bins"], w["queries"], 1003)
    got, st = _run(_material(f), q)
    assert st == 0
    assert np.all(np.isfinite(got))
    idx = np.sort(synth.uniform(9, 9, 200_000) * len(q)).astype(np.int64)
    err, _ = query_error(got[idx], oracle_material(f), q[idx])
    assert err <= QUERY_TOL


def test_multi_material_camera_sweep():
    shapes = [(128, 16, 16), (128, 32, 64), (256, 16, 32), (256, 64, 32), (512, 32, 16),
              (512, 32, 64), (1024, 64, 32), (1024, 16, 64)]
    fs, mats, omats = [], [], []
    for i, (N, R, B) in enumerate(shapes):
        L = int(np.log2(N)) + 1
        f = random_factors(N, L, B, R, 40 + i)
        fs.append(f)
        mats.append(_material(f))
        omats.append(oracle_material(f))
    q = synth.queries_camera([(N, int(np.log2(N)) + 1, B) for N, R, B in shapes], 400_000, 1004)
    for lanes in (None, 8, 32):
        got, st = _run(mats, q, tuning=None if lanes is None else (lanes, 8, 256, 4))
        assert st == 0
        err, _ = query_error(got, omats, q)
        assert err <= QUERY_TOL, lanes


def test_edge_queries():
    f = random_factors(16, 5, 8, 12, 77)
    mat = _material(f)
    om = oracle_material(f)
    rows = [
        (3, 5, 2.0, 1.25, 6.5, 0.5, 8.0, 0),     # plain
        (3, 5, 2.0, 6.5, 1.25, 8.0, 0.5, 0),     # reversed
        (3 - 16 * 7, 5 + 16 * 3, 2.0, 1.25, 6.5, 0.5, 8.0, 0),  # wrap, negative x
        (0, 0, -3.0, 2.0, 2.0, 8.0, 8.0, 0),     # level below 0, zero widths, at B
        (0, 0, 99.0, 0.0, 8.0, 0.0, 8.0, 0),     # level above top, full range
        (1, 2, 3.75, -5.0, 100.0, 3.3, 3.3, 0),  # clamped range, zero-width t
        (1, 2, 0.5, 7.999, 8.0, 0.0, 1e-6, 0),   # tiny widths
    ]
    q = np.array(rows, dtype=synth.QUERY_DTYPE)
    got, st = _run(mat, q)
    assert st == 0
    err, _ = query_error(got, om, q)
    assert err <= QUERY_TOL
    # malformed queries: NaN out and the status bit, neighbours unaffected
    bad = np.array(rows[:3], dtype=synth.QUERY_DTYPE)
    bad[1]["s1"] = np.nan
    bad[2]["material"] = 3
    got, st = _run(mat, bad)
    assert st & 0x2
    assert np.isnan(got[1]) and np.isnan(got[2])
    assert abs(got[0] - oq.cp_range_query(om, bad[:1])[0]) <= 1e-5 * oq.condition_scale(om, bad[:1])[0]


def test_empty_and_ragged_batches():
    import paper_2109_14807_gb300 as g
    f = random_factors(32, 6, 16, 8, 5)
    mat = _material(f)
    empty = torch.empty((0, 8), dtype=torch.int32, device="cuda")
    out = g.range_query(mat, empty)
    assert out.numel() == 0
    for n in (1, 3, 31, 33, 1023):
        q = synth.queries_fractional(32, 6, 16, n, n, frac_level=True)
        got, st = _run(mat, q)
        assert st == 0
        err, _ = query_error(got, oracle_material(f), q)
        assert err <= QUERY_TOL


def test_no_workspace_static_schedule_matches():
    import paper_2109_14807_gb300 as g
    from paper_2109_14807_gb300 import _lib
    f = random_factors(64, 7, 32, 16, 9)
    mat = _material(f)
    q = synth.queries_fractional(64, 7, 32, 20_000, 10)
    qd = g.queries_to_device(q)
    a = g.range_query(mat, qd)
    lib_ = _lib.load()
    out = torch.empty_like(a)
    arr = (_lib.Material * 1)(mat.struct())
    rc = lib_.gsp_range_query(arr, 1, qd.data_ptr(), qd.shape[0], out.data_ptr(), None, None, None,
                              0, torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.equal(a, out)


def test_results_do_not_depend_on_launch_shape():
    # the rank sum has one fixed order, so every tuning gives the same bits
    import paper_2109_14807_gb300 as g
    f = random_factors(128, 8, 32, 64, 21)
    mat = _material(f)
    q = synth.queries_fractional(128, 8, 32, 50_000, 22, frac_level=True)
    qd = g.queries_to_device(q)
    ref = g.range_query(mat, qd, tuning=(32, 8, 256, 4)).clone()
    for tn in [(16, 8, 256, 4), (8, 4, 128, 1), (4, 16, 256, 8), (32, 1, 64, 64), (16, 2, 256, 2)]:
        got = g.range_query(mat, qd, tuning=tn)
        assert torch.equal(got, ref), tn
    f2 = random_factors(64, 7, 16, 37, 23)  # rank not a multiple of 32
    m2 = _material(f2)
    q2 = g.queries_to_device(synth.queries_fractional(64, 7, 16, 20_000, 24, frac_level=True))
    r2 = g.range_query(m2, q2, tuning=(32, 8, 256, 4)).clone()
    for lanes in (4, 8, 16):
        assert torch.equal(g.range_query(m2, q2, tuning=(lanes, 8, 256, 4)), r2), lanes
    # rank 16: runs of 4 (4 lanes), 2 (8 lanes) and single ranks (16, 32 lanes)
    f3 = random_factors(64, 7, 16, 16, 25)
    m3 = _material(f3)
    q3 = g.queries_to_device(synth.queries_fractional(64, 7, 16, 20_000, 26, frac_level=True))
    r3 = g.range_query(m3, q3, tuning=(32, 8, 256, 4)).clone()
    for lanes in (4, 8, 16):
        assert torch.equal(g.range_query(m3, q3, tuning=(lanes, 8, 256, 4)), r3), lanes
    # fx, fy rows 4 bytes off a 16-byte boundary: single-rank loads, same bits
    fd = to_device_factors(f3)
    for k in ("fx", "fy"):
        buf = torch.zeros(fd[k].numel() + 1, dtype=torch.float32, device=fd[k].device)
        buf[1:].copy_(fd[k].reshape(-1))
        fd[k] = buf[1:].view(fd[k].shape)
    m4 = g.QueryMaterial.from_factors(fd)
    g.build_query_tables(m4)
    assert fd["fx"].data_ptr() % 16 != 0
    for lanes in (4, 8):
        assert torch.equal(g.range_query(m4, q3, tuning=(lanes, 8, 256, 4)), r3), lanes


def test_graph_replay_and_autotuner():
    import paper_2109_14807_gb300 as g
    from paper_2109_14807_gb300 import tune
    shapes = [(256, 16, 32), (512, 64, 32)]
    mats = []
    for i, (N, R, B) in enumerate(shapes):
        mats.append(_material(random_factors(N, int(np.log2(N)) + 1, B, R, 70 + i)))
    q = synth.queries_camera([(N, int(np.log2(N)) + 1, B) for N, R, B in shapes], 300_000, 71)
    qd = g.queries_to_device(q)
    tn = tune.autotune_query(mats, qd, sample=100_000, repeats=1, cache_path=None)
    assert len(tn) == 4
    eager = g.range_query(mats, qd, tuning=tn).clone()
    out = torch.empty_like(eager)
    graph = tune.QueryGraph(mats, qd, out, tuning=tn)
    out.zero_()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
    err, _ = query_error(out.cpu().numpy(), [oracle_material(random_factors(N, int(np.log2(N)) + 1, B, R, 70 + i))
                                             for i, (N, R, B) in enumerate(shapes)], q)
    assert err <= QUERY_TOL
