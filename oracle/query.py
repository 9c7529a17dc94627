"""Oracle: CP point and range queries, the dense range average, and the adjoint
(test infrastructure).

A material is a dict of FP64 factor matrices, one row per index, one column
per rank r:  fx [N][R], fy [N][R], flw [L][R] (the level factor with the CP
weights C_r of Eq. 3 folded in, flw = fl * lambda), fs [B][R], ft [B][R].

Query semantics (this library's reading of Sec. 4.3-4.4 and Sec. 5.1):

* x, y are taken modulo N (the map tiles);
* the level is clamped to [0, L-1] (Sec. 5.1 clamps footprints above the
  coarsest level); with l0 = floor(level), f = level - l0 and l1 = min(l0+1, L-1),
  the result blends levels as (1-f) Q(l0) + f Q(l1) (Sec. 4.1, Sec. 4.3:
  linear interpolation between precomputed footprint levels);
* an angular range [s0, s1] x [t0, t1] is in bin units, clamped to [0, B] and
  reordered when reversed; bin k covers [k, k+1).  The range average of a 1D
  factor is its integral over [s0, s1] divided by the width, the factor being
  piecewise constant over bins; a zero-width range is a point query of the bin
  containing s0 (bin B-1 when s0 = B).
"""
from __future__ import annotations

import numpy as np

FACTORS = ("fx", "fy", "flw", "fs", "ft")


def prefix_table(f: np.ndarray) -> np.ndarray:
    """1D summed-area table of Sec. 4.4: P[i] = sum_{k < i} f[k], i = 0..B."""
    P = np.zeros((f.shape[0] + 1,) + f.shape[1:], dtype=np.float64)
    P[1:] = np.cumsum(f, axis=0)
    return P


def normalise_queries(q: np.ndarray, N: int, levels: int, bins: int):
    """Apply the wrap / clamp / reorder rules.  Returns a dict of FP64 / int64
    arrays and a boolean mask of invalid queries (non-finite fields)."""
    lev = q["level"].astype(np.float64)
    s0, s1 = q["s0"].astype(np.float64), q["s1"].astype(np.float64)
    t0, t1 = q["t0"].astype(np.float64), q["t1"].astype(np.float64)
    bad = ~(np.isfinite(lev) & np.isfinite(s0) & np.isfinite(s1) & np.isfinite(t0) & np.isfinite(t1))
    lev = np.where(bad, 0.0, lev)
    lev = np.clip(lev, 0.0, levels - 1)
    l0 = np.floor(lev).astype(np.int64)
    f = lev - l0
    l1 = np.minimum(l0 + 1, levels - 1)
    out = dict(x=q["x"].astype(np.int64) % N, y=q["y"].astype(np.int64) % N,
               l0=l0, l1=l1, f=f)
    for name, a, b in (("s", s0, s1), ("t", t0, t1)):
        a = np.clip(np.where(bad, 0.0, a), 0.0, bins)
        b = np.clip(np.where(bad, 0.0, b), 0.0, bins)
        out[name + "0"], out[name + "1"] = np.minimum(a, b), np.maximum(a, b)
    return out, bad


def range_mean_sat(f: np.ndarray, P: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Average of the piecewise-constant factor f over [a, b] from its 1D SAT:
    (F(b) - F(a)) / (b - a) with F(s) = P[floor s] + (s - floor s) f[floor s]
    (F(B) = P[B]); two table look-ups per endpoint (Sec. 4.4).  Rows: one per
    query; returns [n][R]."""
    B = f.shape[0]

    def F(s):
        k = np.minimum(np.floor(s).astype(np.int64), B)
        frac = (s - k)[:, None]
        fk = np.where((k < B)[:, None], f[np.minimum(k, B - 1)], 0.0)
        return P[k] + frac * fk

    width = b - a
    zero = width <= 0
    safe = np.where(zero, 1.0, width)[:, None]
    avg = (F(b) - F(a)) / safe
    point = f[np.minimum(np.floor(a).astype(np.int64), B - 1)]
    return np.where(zero[:, None], point, avg)


def _material_terms(mat: dict, nq: dict, sel: np.ndarray):
    fx, fy, flw, fs, ft = (np.asarray(mat[k], dtype=np.float64) for k in FACTORS)
    x, y = nq["x"][sel], nq["y"][sel]
    l0, l1, f = nq["l0"][sel], nq["l1"][sel], nq["f"][sel][:, None]
    L = (1.0 - f) * flw[l0] + f * flw[l1]
    S = range_mean_sat(fs, prefix_table(fs), nq["s0"][sel], nq["s1"][sel])
    T = range_mean_sat(ft, prefix_table(ft), nq["t0"][sel], nq["t1"][sel])
    return fx[x], fy[y], L, S, T


def _dims(mat):
    return mat["fx"].shape[0], mat["flw"].shape[0], mat["fs"].shape[0]


def cp_range_query(materials, q: np.ndarray) -> np.ndarray:
    """Eq. 5: sum_r C_r Xbar_r Ybar_r Z_r, extended to this tensor's five modes
    (Appendix: 'extends to higher dimensions'):
    q = sum_r fx[x,r] fy[y,r] ((1-f) flw[l0,r] + f flw[l1,r]) Sbar_r Tbar_r.
    Invalid queries give NaN."""
    if isinstance(materials, dict):
        materials = [materials]
    out = np.full(len(q), np.nan)
    for m, mat in enumerate(materials):
        sel = q["material"] == m
        if not np.any(sel):
            continue
        nq, bad = normalise_queries(q, *_dims(mat))
        X, Y, L, S, T = _material_terms(mat, nq, sel)
        v = np.sum(X * Y * L * S * T, axis=1)
        out[sel] = np.where(bad[sel], np.nan, v)
    return out


def condition_scale(materials, q: np.ndarray) -> np.ndarray:
    """kappa_i = sum_r |fx fy L| * avg|fs| * avg|ft| over the query's ranges: the
    size of the terms the rank sum adds up, so |q - q_ref| / max(|q_ref|, kappa)
    is the rounding error relative to the magnitudes summed."""
    if isinstance(materials, dict):
        materials = [materials]
    out = np.zeros(len(q))
    for m, mat in enumerate(materials):
        sel = q["material"] == m
        if not np.any(sel):
            continue
        absmat = {k: np.abs(np.asarray(mat[k], dtype=np.float64)) for k in FACTORS}
        nq, _ = normalise_queries(q, *_dims(mat))
        X, Y, L, S, T = _material_terms(absmat, nq, sel)
        out[sel] = np.sum(X * Y * L * S * T, axis=1)
    return out


def kappa_relative_error(got, ref, kappa) -> np.ndarray:
    """|got - ref| / max(|ref|, kappa) per query; a query whose reference and
    condition scale are both exactly zero (a range over empty bins) counts as
    exact when got is zero too and as infinitely wrong otherwise."""
    got = np.asarray(got, dtype=np.float64)
    denom = np.maximum(np.abs(ref), kappa)
    diff = np.abs(got - ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        err = diff / denom
    return np.where(denom > 0, err, np.where(diff == 0, 0.0, np.inf))


def cp_point_query(mat: dict, x: int, y: int, l: int, s: int, t: int) -> float:
    """Eq. 4: D(x, y, z) = sum_r C_r X_r(x) Y_r(y) Z_r(z), five integer indices."""
    return float(np.sum(mat["fx"][x] * mat["fy"][y] * mat["flw"][l] * mat["fs"][s] * mat["ft"][t]))


def reconstruct(mat: dict) -> np.ndarray:
    """Dense tensor sum_r fx_r o fy_r o flw_r o fs_r o ft_r, logical order (x, y, l, s, t)."""
    return np.einsum("xr,yr,lr,sr,tr->xylst", mat["fx"], mat["fy"], mat["flw"],
                     mat["fs"], mat["ft"], optimize="greedy")


def overlap_weights(a: float, b: float, bins: int) -> np.ndarray:
    """Length of [k, k+1) inside [a, b] for every bin k, divided by b - a; a
    zero-width range puts weight 1 on the bin holding a (bin B-1 when a = B)."""
    k = np.arange(bins, dtype=np.float64)
    if b <= a:
        w = np.zeros(bins)
        w[min(int(np.floor(a)), bins - 1)] = 1.0
        return w
    return np.clip(np.minimum(k + 1.0, b) - np.maximum(k, a), 0.0, None) / (b - a)


def dense_range_query(T_log: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Brute-force range average over a dense tensor (x, y, l, s, t): the
    overlap-weighted mean of all bins of the rectangle, blended across levels.
    With integer endpoints this is the plain mean of Appendix Eq. (M*N terms)."""
    N, _, levels, bins, _ = T_log.shape
    nq, bad = normalise_queries(q, N, levels, bins)
    out = np.empty(len(q))
    for i in range(len(q)):
        if bad[i]:
            out[i] = np.nan
            continue
        ws = overlap_weights(nq["s0"][i], nq["s1"][i], bins)
        wt = overlap_weights(nq["t0"][i], nq["t1"][i], bins)
        x, y, f = nq["x"][i], nq["y"][i], nq["f"][i]
        q0 = ws @ T_log[x, y, nq["l0"][i]] @ wt
        q1 = ws @ T_log[x, y, nq["l1"][i]] @ wt
        out[i] = (1.0 - f) * q0 + f * q1
    return out


def cp_range_query_adjoint(materials, q: np.ndarray, g: np.ndarray):
    """Gradients of sum_i g_i q_i with respect to every factor of every material
    (list of dicts with keys of FACTORS), differentiating the range query above
    directly: the range average is linear in fs with weights overlap_weights."""
    single = isinstance(materials, dict)
    if single:
        materials = [materials]
    grads = []
    g = np.asarray(g, dtype=np.float64)
    for m, mat in enumerate(materials):
        N, levels, bins = _dims(mat)
        G = {k: np.zeros_like(np.asarray(mat[k], dtype=np.float64)) for k in FACTORS}
        grads.append(G)
        sel = np.nonzero((q["material"] == m))[0]
        if len(sel) == 0:
            continue
        nq, bad = normalise_queries(q, N, levels, bins)
        fx, fy, flw, fs, ft = (np.asarray(mat[k], dtype=np.float64) for k in FACTORS)
        for i in sel:
            if bad[i]:
                continue
            x, y, l0, l1, f = nq["x"][i], nq["y"][i], nq["l0"][i], nq["l1"][i], nq["f"][i]
            ws = overlap_weights(nq["s0"][i], nq["s1"][i], bins)
            wt = overlap_weights(nq["t0"][i], nq["t1"][i], bins)
            L = (1.0 - f) * flw[l0] + f * flw[l1]
            S = ws @ fs
            T = wt @ ft
            gi = g[i]
            G["fx"][x] += gi * fy[y] * L * S * T
            G["fy"][y] += gi * fx[x] * L * S * T
            G["flw"][l0] += gi * (1.0 - f) * fx[x] * fy[y] * S * T
            G["flw"][l1] += gi * f * fx[x] * fy[y] * S * T
            G["fs"] += gi * np.outer(ws, fx[x] * fy[y] * L * T)
            G["ft"] += gi * np.outer(wt, fx[x] * fy[y] * L * S)
    return grads[0] if single else grads


def cp_range_query_interp(materials, q: np.ndarray) -> np.ndarray:
    """Range queries at fractional texel positions (Sec. 4.1: interpolation
    between neighbouring footprint samples), by definition the bilinear blend
    sum_{i,j in {0,1}} w_i(x) w_j(y) Q(floor(x) + i, floor(y) + j) of the
    integer-position range queries (positions mod N)."""
    x = q["x"].astype(np.float64)
    y = q["y"].astype(np.float64)
    x0, y0 = np.floor(x), np.floor(y)
    wx, wy = x - x0, y - y0
    out = np.zeros(len(q))
    for i in (0, 1):
        for j in (0, 1):
            qi = np.zeros(len(q), dtype=[(k, q.dtype[k] if k not in ("x", "y") else "<i4")
                                         for k in q.dtype.names])
            for k in q.dtype.names:
                if k not in ("x", "y"):
                    qi[k] = q[k]
            qi["x"] = (x0 + i).astype(np.int64)
            qi["y"] = (y0 + j).astype(np.int64)
            w = (wx if i else 1.0 - wx) * (wy if j else 1.0 - wy)
            out += w * cp_range_query(materials, qi)
    return out


def sg_support_angle(amplitude: np.ndarray, sharpness: np.ndarray, eps: float = 0.3) -> np.ndarray:
    """Compact-eps support of a spherical Gaussian A exp(lambda (cos v - 1))
    (Sec. 5.4): the angle theta inside which the lobe exceeds eps,
    theta = arccos((ln eps - ln A) / lambda + 1); pi when the argument is below
    -1 (the whole sphere), 0 when A <= eps (nowhere)."""
    A = np.asarray(amplitude, dtype=np.float64)
    lam = np.asarray(sharpness, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        c = (np.log(eps) - np.log(A)) / lam + 1.0
    theta = np.arccos(np.clip(c, -1.0, 1.0))
    return np.where(A > eps, theta, 0.0)


def env_queries(sgs: np.ndarray, records: np.ndarray, bins, eps: float = 0.3) -> np.ndarray:
    """Range-query descriptors of Sec. 5.4 for shading records: the square of
    side Q = B theta / pi (the paper's 256-pixel image -> B bins) centred on
    the bin of the half vector h = normalize(wo + axis).  `bins[m]` is the bin
    count of material m.  Returns a structured array of queries (FP64 ends)."""
    bins = np.asarray(bins)
    g = sgs[records["sg"]]
    B = bins[records["material"]].astype(np.float64)
    h = records["wo"].astype(np.float64) + g["axis"].astype(np.float64)
    h = h / np.linalg.norm(h, axis=1)[:, None]
    theta = sg_support_angle(g["amplitude"], g["sharpness"], eps)
    side = B * theta / np.pi
    sc, tc = (h[:, 0] + 1.0) * B / 2, (h[:, 1] + 1.0) * B / 2
    q = np.zeros(len(records), dtype=[("x", "<i8"), ("y", "<i8"), ("level", "<f8"), ("s0", "<f8"),
                                      ("s1", "<f8"), ("t0", "<f8"), ("t1", "<f8"), ("material", "<u4")])
    q["x"], q["y"], q["level"], q["material"] = records["x"], records["y"], records["level"], records["material"]
    q["s0"], q["s1"], q["t0"], q["t1"] = sc - side / 2, sc + side / 2, tc - side / 2, tc + side / 2
    return q
