"""Pins of the fractional-position range query (Sec. 4.1 interpolation
between neighbouring footprints): integer positions reduce to the plain range
query, the blend equals one query with interpolated factor rows (the CP tensor
is multilinear), and it equals the bilinear blend of brute-force range
averages of the dense reconstruction."""
import numpy as np

import synth
from oracle import query as oq


def _material(N, L, B, R, seed):
    return {k: 2 * synth.uniform(seed, 70 + i, n * R).reshape(n, R) - 1
            for i, (k, n) in enumerate((("fx", N), ("fy", N), ("flw", L), ("fs", B), ("ft", B)))}


def test_integer_positions_are_plain_queries():
    mat = _material(16, 5, 8, 4, 1)
    qi = synth.queries_fractional(16, 5, 8, 200, 3, frac_level=True)
    qf = np.zeros(len(qi), dtype=synth.QUERY_F_DTYPE)
    for k in qi.dtype.names:
        qf[k] = qi[k]
    assert np.allclose(oq.cp_range_query_interp(mat, qf), oq.cp_range_query(mat, qi), rtol=0, atol=1e-14)


def test_blend_equals_interpolated_factor_rows():
    N, L, B = 16, 5, 8
    mat = _material(N, L, B, 4, 2)
    q = synth.queries_fractional_xy(N, L, B, 300, 5)
    got = oq.cp_range_query_interp(mat, q)
    x0, y0 = np.floor(q["x"].astype(np.float64)), np.floor(q["y"].astype(np.float64))
    wx, wy = q["x"] - x0, q["y"] - y0
    ix, iy = x0.astype(np.int64), y0.astype(np.int64)
    fx = (1 - wx)[:, None] * mat["fx"][ix % N] + wx[:, None] * mat["fx"][(ix + 1) % N]
    fy = (1 - wy)[:, None] * mat["fy"][iy % N] + wy[:, None] * mat["fy"][(iy + 1) % N]
    qq = np.zeros(len(q), dtype=synth.QUERY_DTYPE)
    for k in ("level", "s0", "s1", "t0", "t1"):
        qq[k] = q[k]
    ref = np.empty(len(q))
    for i in range(len(q)):  # one-texel material holding the interpolated rows
        m1 = dict(fx=fx[i:i + 1], fy=fy[i:i + 1], flw=mat["flw"], fs=mat["fs"], ft=mat["ft"])
        ref[i] = oq.cp_range_query(m1, qq[i:i + 1])[0]
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_blend_of_dense_range_averages():
    N, L, B = 8, 4, 8
    mat = _material(N, L, B, 3, 4)
    T = oq.reconstruct(mat)
    q = synth.queries_fractional_xy(N, L, B, 100, 6)
    got = oq.cp_range_query_interp(mat, q)
    ref = np.zeros(len(q))
    x0, y0 = np.floor(q["x"].astype(np.float64)), np.floor(q["y"].astype(np.float64))
    for i in (0, 1):
        for j in (0, 1):
            qi = np.zeros(len(q), dtype=synth.QUERY_DTYPE)
            for k in ("level", "s0", "s1", "t0", "t1"):
                qi[k] = q[k]
            qi["x"] = (x0 + i).astype(np.int64) % N
            qi["y"] = (y0 + j).astype(np.int64) % N
            w = np.where(i, q["x"] - x0, 1 - (q["x"] - x0)) * np.where(j, q["y"] - y0, 1 - (q["y"] - y0))
            ref += w * oq.dense_range_query(T, qi)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-13)
