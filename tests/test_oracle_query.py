"""Pins for the oracle's point / range queries and adjoint (Sec. 4.3-4.4, Appendix)."""
import os

import numpy as np
import pytest

import synth
from oracle import query as oq

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _material(N, L, B, R, seed, signed=True):
    u = synth.uniform(seed, 5, (2 * N + L + 2 * B) * R)
    if signed:
        u = 2.0 * u - 1.0
    off, mat = 0, {}
    for k, n in (("fx", N), ("fy", N), ("flw", L), ("fs", B), ("ft", B)):
        mat[k] = u[off:off + n * R].reshape(n, R)
        off += n * R
    return mat


def _queries(rows):
    q = np.zeros(len(rows), dtype=synth.QUERY_DTYPE)
    for i, (x, y, lev, s0, s1, t0, t1) in enumerate(rows):
        q[i] = (x, y, lev, s0, s1, t0, t1, 0)
    return q


def test_golden_rank2_hand_worked():
    mat = dict(fx=np.array([[1, 1], [3, -1]], float), fy=np.array([[2, 1], [1, 1]], float),
               flw=np.array([[0.5, 1], [1.5, 2]], float),
               fs=np.array([[1, 0], [2, 1], [3, 0], [4, 1]], float),
               ft=np.array([[4, 1], [0, 1], [2, 1], [2, 1]], float))
    rows = np.loadtxt(os.path.join(GOLDEN, "range_query_rank2.txt"), comments="#")
    q = _queries([tuple(r[:7]) for r in rows])
    got = oq.cp_range_query(mat, q)
    assert np.allclose(got, rows[:, 7], rtol=0, atol=1e-14)
    dense = oq.dense_range_query(oq.reconstruct(mat), q)
    assert np.allclose(dense, rows[:, 7], rtol=0, atol=1e-13)


@pytest.mark.parametrize("R", [1, 3, 8])
def test_appendix_proposition_sat_equals_dense(R):
    # CP range query through 1D SATs == brute-force rectangle average of the
    # dense reconstruction, for fractional ranges and levels (Appendix, Eq. 5)
    N, L, B = 4, 3, 8
    mat = _material(N, L, B, R, 10 + R)
    q = synth.queries_fractional(N, L, B, 300, 77 + R, wmin=0.01, wmax=8.0, frac_level=True)
    got = oq.cp_range_query(mat, q)
    ref = oq.dense_range_query(oq.reconstruct(mat), q)
    kappa = oq.condition_scale(mat, q)
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), kappa)) < 1e-12


def test_integer_range_equals_mean_of_point_queries():
    # Fig. 7: range query == average of point queries over the rectangle
    N, L, B, R = 4, 3, 8, 5
    mat = _material(N, L, B, R, 3)
    q = synth.queries_integer(N, L, B, 60, 5)
    got = oq.cp_range_query(mat, q)
    for i in range(len(q)):
        x, y, l = int(q["x"][i]), int(q["y"][i]), int(q["level"][i])
        s0, s1, t0, t1 = (int(q[k][i]) for k in ("s0", "s1", "t0", "t1"))
        pts = [oq.cp_point_query(mat, x, y, l, s, t) for s in range(s0, s1) for t in range(t0, t1)]
        assert abs(got[i] - np.mean(pts)) <= 1e-12 * max(1.0, np.max(np.abs(pts)))


def test_zero_width_is_point_query_and_reconstruction_entry():
    N, L, B, R = 4, 3, 8, 4
    mat = _material(N, L, B, R, 4)
    X = oq.reconstruct(mat)
    rng_rows = []
    for (x, y, l, s, t) in [(0, 0, 0, 0, 0), (3, 2, 2, 7, 1), (1, 3, 1, 4, 4)]:
        rng_rows.append((x, y, l, s + 0.25, s + 0.25, t + 0.75, t + 0.75))
    got = oq.cp_range_query(mat, _queries(rng_rows))
    for i, (x, y, l, s, t) in enumerate([(0, 0, 0, 0, 0), (3, 2, 2, 7, 1), (1, 3, 1, 4, 4)]):
        p = oq.cp_point_query(mat, x, y, l, s, t)
        assert abs(got[i] - p) < 1e-14
        assert abs(X[x, y, l, s, t] - p) < 1e-14  # Sec. 4.3: exact as the full image


def test_sat_prefix_difference_is_direct_sum():
    f = synth.uniform(1, 2, 40).reshape(10, 4) - 0.5
    P = oq.prefix_table(f)
    for a in range(11):
        for b in range(a, 11):
            assert np.allclose(P[b] - P[a], f[a:b].sum(axis=0), atol=1e-15)


def test_degenerate_queries():
    N, L, B, R = 4, 3, 8, 3
    mat = _material(N, L, B, R, 9)
    base = _queries([(1, 2, 1.5, 2.25, 5.5, 0.5, 7.0)])
    ref = oq.cp_range_query(mat, base)[0]
    # reversed rectangle
    assert oq.cp_range_query(mat, _queries([(1, 2, 1.5, 5.5, 2.25, 7.0, 0.5)]))[0] == ref
    # wrapped spatial index
    assert oq.cp_range_query(mat, _queries([(1 + 4 * N, 2 - 3 * N, 1.5, 2.25, 5.5, 0.5, 7.0)]))[0] == ref
    # out-of-range ends are clamped to [0, B]
    a = oq.cp_range_query(mat, _queries([(1, 2, 1.0, -3.0, 99.0, 0.0, 8.0)]))[0]
    b = oq.cp_range_query(mat, _queries([(1, 2, 1.0, 0.0, 8.0, 0.0, 8.0)]))[0]
    assert a == b
    # level clamp below and above
    lo = oq.cp_range_query(mat, _queries([(0, 0, -2.0, 1, 2, 1, 2)]))[0]
    assert lo == oq.cp_point_query(mat, 0, 0, 0, 1, 1)
    hi = oq.cp_range_query(mat, _queries([(0, 0, 50.0, 1, 2, 1, 2)]))[0]
    assert hi == oq.cp_point_query(mat, 0, 0, L - 1, 1, 1)
    # full range == mean over all bins
    full = oq.cp_range_query(mat, _queries([(3, 3, 2, 0, B, 0, B)]))[0]
    X = oq.reconstruct(mat)
    assert abs(full - X[3, 3, 2].mean()) < 1e-14
    # non-finite field -> NaN
    q = _queries([(0, 0, 0, 0, 1, 0, 1)])
    q["s1"] = np.nan
    assert np.isnan(oq.cp_range_query(mat, q)[0])


def test_multi_material_routing():
    m0, m1 = _material(4, 3, 8, 2, 1), _material(8, 4, 4, 3, 2)
    q0 = synth.queries_fractional(4, 3, 8, 20, 3, frac_level=True)
    q1 = synth.queries_fractional(8, 4, 4, 20, 4, frac_level=True, material=1)
    q = np.concatenate([q0, q1])
    both = oq.cp_range_query([m0, m1], q)
    assert np.array_equal(both[:20], oq.cp_range_query(m0, q0))
    q1m = q1.copy()
    q1m["material"] = 0
    assert np.array_equal(both[20:], oq.cp_range_query(m1, q1m))


def test_adjoint_matches_central_differences():
    N, L, B, R = 4, 3, 8, 3
    mat = _material(N, L, B, R, 21)
    q = synth.queries_fractional(N, L, B, 25, 8, wmin=0.01, wmax=8.0, frac_level=True)
    q[3]["s1"] = q[3]["s0"]  # one zero-width range
    g = synth.uniform(3, 3, len(q)) - 0.5
    G = oq.cp_range_query_adjoint(mat, q, g)
    # q is linear in every single factor entry, so a central difference is exact
    # up to rounding for any step; a moderate step keeps rounding small
    h = 1e-3
    for k in oq.FACTORS:
        for idx in np.ndindex(*mat[k].shape):
            plus = {kk: vv.copy() for kk, vv in mat.items()}
            minus = {kk: vv.copy() for kk, vv in mat.items()}
            plus[k][idx] += h
            minus[k][idx] -= h
            fd = (g @ oq.cp_range_query(plus, q) - g @ oq.cp_range_query(minus, q)) / (2 * h)
            assert abs(fd - G[k][idx]) <= 1e-9 * max(1.0, abs(fd)), (k, idx, fd, G[k][idx])


def test_adjoint_is_transpose_of_linear_map_in_fs():
    # q is linear in fs: sum_i g_i q_i(fs) == <G_fs, fs> exactly when only fs varies
    N, L, B, R = 4, 2, 8, 2
    mat = _material(N, L, B, R, 5)
    q = synth.queries_fractional(N, L, B, 30, 6, frac_level=True)
    g = synth.uniform(1, 1, len(q))
    G = oq.cp_range_query_adjoint(mat, q, g)
    assert abs(g @ oq.cp_range_query(mat, q) - np.sum(G["fs"] * mat["fs"])) < 1e-12


def test_kappa_relative_error_zero_scale():
    got = np.array([0.0, 1e-3, 2.0, 0.0])
    ref = np.array([0.0, 0.0, 2.0 + 1e-6, 0.0])
    kap = np.array([0.0, 0.0, 4.0, 1.0])
    e = oq.kappa_relative_error(got, ref, kap)
    assert e[0] == 0.0 and np.isinf(e[1]) and abs(e[2] - 1e-6 / 4.0) < 1e-15 and e[3] == 0.0
