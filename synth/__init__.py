"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module holds no arithmetic of the method itself (no binning, no footprint
sums, no tensor decomposition, no queries).  It only draws random numbers and
shapes them into the inputs the method consumes:

* tileable normal maps, stored as FP32 (n.x, n.y) pairs, row-major [y][x][2];
  n.z is implied positive (the maps stand in for the metallic-flake and
  brushed-metal normal maps of Sec. 6, Tab. 2, which are not available);
* initial CP factors for ALS (the paper does not say how ALS is initialised);
* batches of 32-byte range-query descriptors.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014) used as a
counter-based generator: output i of stream k under seed s is
``mix(key(s, k) + (i + 1) * 0x9E3779B97F4A7C15)``, the standard SplitMix64
sequence started from the state ``key(s, k)``.  Normal deviates use the
Box-Muller transform.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "QUERY_DTYPE", "SAMPLE_DTYPE", "splitmix64", "uniform", "normal", "flake_map", "brushed_map",
    "sample_footprints", "sample_uniforms", "QUERY_F_DTYPE", "queries_fractional_xy",
    "SG_DTYPE", "ENV_RECORD_DTYPE", "env_lobes", "env_records",
    "init_factors", "queries_integer", "queries_fractional", "queries_camera",
    "WORKLOADS",
    "cluster_init",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# 32-byte query descriptor: {int32 x, y; float level, s0, s1, t0, t1; uint32 material}
QUERY_DTYPE = np.dtype([
    ("x", "<i4"), ("y", "<i4"), ("level", "<f4"),
    ("s0", "<f4"), ("s1", "<f4"), ("t0", "<f4"), ("t1", "<f4"),
    ("material", "<u4"),
])
assert QUERY_DTYPE.itemsize == 32

# A range query at a fractional texel position (same layout, float x, y).
QUERY_F_DTYPE = np.dtype([
    ("x", "<f4"), ("y", "<f4"), ("level", "<f4"),
    ("s0", "<f4"), ("s1", "<f4"), ("t0", "<f4"), ("t1", "<f4"),
    ("material", "<u4"),
])
assert QUERY_F_DTYPE.itemsize == 32

# A spherical Gaussian lobe of an environment light and a shading record
# choosing one (32 bytes each).
SG_DTYPE = np.dtype([("axis", "<f4", (3,)), ("amplitude", "<f4"), ("sharpness", "<f4"),
                     ("pad", "<f4", (3,))])
ENV_RECORD_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("level", "<f4"), ("wo", "<f4", (3,)),
                             ("sg", "<u4"), ("material", "<u4")])
assert SG_DTYPE.itemsize == 32 and ENV_RECORD_DTYPE.itemsize == 32

# Footprint of a hierarchical NDF sample: texel, level, material (16 bytes).
SAMPLE_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("level", "<f4"), ("material", "<u4")])
assert SAMPLE_DTYPE.itemsize == 16


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to state+gamma (vectorised, wraps mod 2^64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([(int(seed) & 0xFFFFFFFFFFFFFFFF) ^ ((int(stream) & 0xFFFFFF) << 40)],
                 dtype=np.uint64)
    return splitmix64(s)[0]


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n float64 draws in [0, 1) with 53 random bits each."""
    idx = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = _key(seed, stream) + idx * _GAMMA
    bits = splitmix64(state) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal deviates by Box-Muller (one deviate per pair of uniforms)."""
    u = uniform(seed, stream, 2 * n)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def _slopes_to_normals(p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Surface slopes (dz/dx, dz/dy) -> FP32 (n.x, n.y) of n = normalise(-p, -q, 1)."""
    inv = 1.0 / np.sqrt(p * p + q * q + 1.0)
    out = np.empty(p.shape + (2,), dtype=np.float32)
    out[..., 0] = (-p * inv).astype(np.float32)
    out[..., 1] = (-q * inv).astype(np.float32)
    return out


def _torus_nearest(sites: np.ndarray, N: int) -> np.ndarray:
    """Index of the nearest site to every texel centre on the N x N torus."""
    yy, xx = np.meshgrid(np.arange(N) + 0.5, np.arange(N) + 0.5, indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
    if len(sites) * N * N <= 1 << 22:
        d = pts[:, None, :] - sites[None, :, :]
        d = np.abs(d)
        d = np.minimum(d, N - d)
        dist = (d * d).sum(-1)
        idx = np.argmin(dist, axis=1)  # ties -> lowest index
    else:
        from scipy.spatial import cKDTree
        tree = cKDTree(np.mod(sites, N), boxsize=float(N))
        _, idx = tree.query(pts, k=1)
    return idx.reshape(N, N)


def flake_map(N: int, cells: int, alpha: float, seed: int) -> np.ndarray:
    """Voronoi metallic flakes: `cells` sites uniform on the N x N torus; every
    texel takes its nearest site's normal; per-cell slopes are iid
    N(0, alpha^2 / 2) per axis (the Beckmann slope variance).  Returns FP32
    [N][N][2] = (n.x, n.y), indexed [y][x]."""
    u = uniform(seed, 1, 2 * cells) * N
    sites = np.stack([u[0::2], u[1::2]], axis=1)
    cell = _torus_nearest(sites, N)
    sd = alpha / math.sqrt(2.0)
    p = normal(seed, 2, cells) * sd
    q = normal(seed, 3, cells) * sd
    return _slopes_to_normals(p[cell], q[cell])


def brushed_map(N: int, sigma_x: float, sigma_y: float, n_scratch: int, seed: int,
                scratch_slope: float = 0.5) -> np.ndarray:
    """Brushed metal: per-texel iid slopes p ~ N(0, sigma_x^2), q ~ N(0, sigma_y^2),
    overdrawn by `n_scratch` one-texel-wide line segments on the torus (length
    U[N/8, N/2], random direction) whose slope is `scratch_slope` perpendicular
    to the segment, sign chosen per scratch."""
    p = normal(seed, 1, N * N).reshape(N, N) * sigma_x
    q = normal(seed, 2, N * N).reshape(N, N) * sigma_y
    u = uniform(seed, 3, 6 * n_scratch).reshape(n_scratch, 6)
    for k in range(n_scratch):
        x0, y0 = u[k, 0] * N, u[k, 1] * N
        th = u[k, 2] * math.pi
        length = N / 8 + u[k, 3] * (N / 2 - N / 8)
        sign = 1.0 if u[k, 4] < 0.5 else -1.0
        c, s = math.cos(th), math.sin(th)
        steps = np.arange(int(math.ceil(length * 4)) + 1) * 0.25
        xs = np.floor(x0 + steps * c).astype(np.int64) % N
        ys = np.floor(y0 + steps * s).astype(np.int64) % N
        p[ys, xs] = sign * scratch_slope * (-s)
        q[ys, xs] = sign * scratch_slope * c
    return _slopes_to_normals(p, q)


def init_factors(N: int, levels: int, bins: int, rank: int, seed: int) -> dict:
    """Seeded U[0,1) initial factors, filled in the order fx, fy, fl, fs, ft, each
    row-major [rows][rank], from one stream.  Returned as float64 (the oracle's
    precision); the FP32 copies handed to the GPU are exact roundings of these."""
    shapes = [("fx", N), ("fy", N), ("fl", levels), ("fs", bins), ("ft", bins)]
    total = sum(n for _, n in shapes) * rank
    u = uniform(seed, 7, total)
    out, off = {}, 0
    for name, n in shapes:
        out[name] = u[off:off + n * rank].reshape(n, rank).copy()
        off += n * rank
    return out


def cluster_init(G: int, offsets: np.ndarray, rank: int, seed: int, block: int = 16):
    """Seeded U[0,1) initial factors of every group of a clustered layout:
    X0, Y0 [G][block][rank] and Z0 [total][rank] (float64; the GPU gets exact
    FP32 roundings).  Group j's rows are drawn from its own stream, so they do
    not depend on the other groups."""
    offsets = np.asarray(offsets, dtype=np.int64)
    X0 = np.empty((G, block, rank))
    Y0 = np.empty((G, block, rank))
    Z0 = np.empty((int(offsets[-1]), rank))
    for j in range(G):
        m = int(offsets[j + 1] - offsets[j])
        u = uniform(seed, 1_000_000 + j, (2 * block + m) * rank)
        X0[j] = u[:block * rank].reshape(block, rank)
        Y0[j] = u[block * rank:2 * block * rank].reshape(block, rank)
        Z0[offsets[j]:offsets[j + 1]] = u[2 * block * rank:].reshape(m, rank)
    return (X0.astype(np.float32).astype(np.float64), Y0.astype(np.float32).astype(np.float64),
            Z0.astype(np.float32).astype(np.float64))


def _empty_queries(n: int) -> np.ndarray:
    return np.zeros(n, dtype=QUERY_DTYPE)


def queries_integer(N: int, levels: int, bins: int, n: int, seed: int,
                    material: int = 0) -> np.ndarray:
    """Uniform queries with integer-aligned bin rectangles: x, y ~ U{0..N-1},
    level ~ U{0..levels-1}, s0 ~ U{0..B-1}, s1 ~ U{s0+1..B}; t likewise."""
    u = uniform(seed, 11, 7 * n).reshape(n, 7)
    q = _empty_queries(n)
    q["x"] = np.minimum((u[:, 0] * N).astype(np.int64), N - 1)
    q["y"] = np.minimum((u[:, 1] * N).astype(np.int64), N - 1)
    q["level"] = np.minimum((u[:, 2] * levels).astype(np.int64), levels - 1)
    s0 = np.minimum((u[:, 3] * bins).astype(np.int64), bins - 1)
    s1 = s0 + 1 + np.minimum((u[:, 4] * (bins - s0)).astype(np.int64), bins - s0 - 1)
    t0 = np.minimum((u[:, 5] * bins).astype(np.int64), bins - 1)
    t1 = t0 + 1 + np.minimum((u[:, 6] * (bins - t0)).astype(np.int64), bins - t0 - 1)
    q["s0"], q["s1"], q["t0"], q["t1"] = s0, s1, t0, t1
    q["material"] = material
    return q


def queries_fractional(N: int, levels: int, bins: int, n: int, seed: int,
                       wmin: float = 0.5, wmax: float = 16.0, frac_level: bool = False,
                       material: int = 0) -> np.ndarray:
    """Uniform queries with fractional bin rectangles: widths log-uniform in
    [wmin, wmax] bins, s0 ~ U[0, B - w], s1 = s0 + w, t drawn independently;
    level ~ U{0..levels-1} (or U[0, levels-1] when `frac_level`)."""
    u = uniform(seed, 12, 7 * n).reshape(n, 7)
    q = _empty_queries(n)
    q["x"] = np.minimum((u[:, 0] * N).astype(np.int64), N - 1)
    q["y"] = np.minimum((u[:, 1] * N).astype(np.int64), N - 1)
    if frac_level:
        q["level"] = (u[:, 2] * (levels - 1)).astype(np.float32)
    else:
        q["level"] = np.minimum((u[:, 2] * levels).astype(np.int64), levels - 1)
    wmax = min(wmax, float(bins))
    lw0, lw1 = math.log(wmin), math.log(wmax)
    for col, (a, b) in (("s", (3, 4)), ("t", (5, 6))):
        w = np.exp(lw0 + u[:, a] * (lw1 - lw0))
        lo = (u[:, b] * (bins - w)).astype(np.float32)
        hi = (lo.astype(np.float64) + w).astype(np.float32)
        hi = np.minimum(hi, np.float32(bins))
        q[col + "0"], q[col + "1"] = lo, hi
    q["material"] = material
    return q


def queries_camera(materials: list, n: int, seed: int) -> np.ndarray:
    """Camera-sweep queries over several materials.  A square pixel raster is cut
    into len(materials) vertical screen regions, one material per region, so
    consecutive queries hit neighbouring texels of one material.  Distance d is
    log-uniform in [1, 2^10] and varies smoothly across the screen;
    level = clamp(log2 d, 0, levels-1) as a float.  Angular widths: 70 % in
    [0.5, 1] bins (point light), 30 % log-uniform in [1, 16] bins (area or
    environment light); centres ~ N(B/2, B/8).  `materials` is a list of
    (N, levels, bins) tuples."""
    m = len(materials)
    side = int(math.ceil(math.sqrt(n)))
    idx = np.arange(n, dtype=np.int64)
    py, px = idx // side, idx % side
    region = np.minimum(px * m // side, m - 1)
    u = uniform(seed, 13, 6 * n).reshape(n, 6)
    g = normal(seed, 14, 2 * n).reshape(n, 2)
    # smooth distance field across the screen plus a little jitter
    phase = (px / side) * 2.0 * math.pi + (py / side) * math.pi
    logd = (0.5 + 0.45 * np.sin(phase) + 0.05 * (u[:, 0] - 0.5)) * 10.0
    logd = np.clip(logd, 0.0, 10.0)
    q = _empty_queries(n)
    Ns = np.array([mt[0] for mt in materials])
    Ls = np.array([mt[1] for mt in materials])
    Bs = np.array([mt[2] for mt in materials], dtype=np.float64)
    Nm, Lm, Bm = Ns[region], Ls[region], Bs[region]
    # texel coordinates follow the pixel raster (scaled by distance)
    q["x"] = (px * (1 + (logd.astype(np.int64) // 3))) % Nm
    q["y"] = (py * (1 + (logd.astype(np.int64) // 3))) % Nm
    q["level"] = np.minimum(logd, Lm - 1).astype(np.float32)
    point = u[:, 1] < 0.7
    w_point = 0.5 + 0.5 * u[:, 2]
    w_area = np.exp(math.log(16.0) * u[:, 3])
    w = np.where(point, w_point, w_area)
    w = np.minimum(w, Bm)
    for col, gi, ui in (("s", 0, 4), ("t", 1, 5)):
        c = Bm / 2 + g[:, gi] * Bm / 8
        lo = np.clip(c - w / 2, 0.0, Bm - w)
        q[col + "0"] = lo.astype(np.float32)
        q[col + "1"] = np.minimum(lo + w, Bm).astype(np.float32)
    q["material"] = region.astype(np.uint32)
    return q


# Workload shapes (map side N, levels L1 = log2 N + 1, bins B, rank R), named by
# what they are.  Seeds: map seed c, query seed 1000 + c, init seed 2000 + c.
WORKLOADS = {
    "flakes32": dict(N=32, levels=6, bins=16, rank=8, seed=1, map="flakes",
                     cells=64, alpha=0.15, sweeps=20, queries=10_000, qkind="integer"),
    "brushed512": dict(N=512, levels=10, bins=32, rank=32, seed=2, map="brushed",
                       sigma_x=0.05, sigma_y=0.3, scratches=200, sweeps=20),
    "flakes1024": dict(N=1024, levels=11, bins=32, rank=64, seed=3, map="flakes",
                       cells=16384, alpha=0.1, queries=10_000_000, qkind="fractional"),
    "clustered256": dict(N=256, levels=9, bins=64, rank=16, seed=6, map="flakes",
                         cells=1024, alpha=0.15, queries=1_000_000, qkind="fractional"),
    "clustered64": dict(N=64, levels=7, bins=64, rank=16, seed=7, map="flakes",
                        cells=64, alpha=0.15, queries=100_000, qkind="fractional"),
    "flakes256": dict(N=256, levels=9, bins=32, rank=16, seed=5, map="flakes",
                      cells=1024, alpha=0.15, sweeps=20, queries=1_000_000,
                      qkind="fractional"),
}


def make_map(w: dict) -> np.ndarray:
    """Normal map for a workload entry of WORKLOADS."""
    if w["map"] == "flakes":
        return flake_map(w["N"], w["cells"], w["alpha"], w["seed"])
    return brushed_map(w["N"], w["sigma_x"], w["sigma_y"], w["scratches"], w["seed"])


def sample_footprints(N: int, levels: int, n: int, seed: int, material: int = 0) -> np.ndarray:
    """Footprints to sample: x, y ~ U{0..N-1}, level ~ U[0, levels-1]."""
    u = uniform(seed, 15, 3 * n).reshape(n, 3)
    s = np.zeros(n, dtype=SAMPLE_DTYPE)
    s["x"] = np.minimum((u[:, 0] * N).astype(np.int64), N - 1)
    s["y"] = np.minimum((u[:, 1] * N).astype(np.int64), N - 1)
    s["level"] = (u[:, 2] * (levels - 1)).astype(np.float32)
    s["material"] = material
    return s


def sample_uniforms(seed: int, n: int, k: int = 8) -> np.ndarray:
    """[n][k] float32 uniforms in [0, 1) for the samplers (float64 draws rounded
    to float32 and kept below 1)."""
    u = uniform(seed, 16, n * k).astype(np.float32)
    return np.minimum(u, np.float32(1.0 - 2.0 ** -24)).reshape(n, k)


def queries_fractional_xy(N: int, levels: int, bins: int, n: int, seed: int,
                          material: int = 0) -> np.ndarray:
    """Queries at fractional texel positions: x, y ~ U[-N, 2N) (exercising the
    wrap), fractional levels and fractional bin rectangles as in
    queries_fractional."""
    base = queries_fractional(N, levels, bins, n, seed, frac_level=True, material=material)
    u = uniform(seed, 17, 2 * n).reshape(n, 2)
    q = np.zeros(n, dtype=QUERY_F_DTYPE)
    for k in ("level", "s0", "s1", "t0", "t1", "material"):
        q[k] = base[k]
    q["x"] = (u[:, 0] * 3 * N - N).astype(np.float32)
    q["y"] = (u[:, 1] * 3 * N - N).astype(np.float32)
    return q


def _hemisphere(u1, u2):
    """Unit vectors uniform on the upper hemisphere (z >= 0)."""
    z = u1
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = 2.0 * math.pi * u2
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def env_lobes(n: int, seed: int) -> np.ndarray:
    """SG lobes of an environment light: axes uniform on the upper hemisphere,
    amplitude log-uniform in [0.1, 10], sharpness log-uniform in [1, 1000]."""
    u = uniform(seed, 18, 4 * n).reshape(n, 4)
    g = np.zeros(n, dtype=SG_DTYPE)
    g["axis"] = _hemisphere(u[:, 0], u[:, 1]).astype(np.float32)
    g["amplitude"] = np.exp(math.log(0.1) + u[:, 2] * math.log(100.0)).astype(np.float32)
    g["sharpness"] = np.exp(u[:, 3] * math.log(1000.0)).astype(np.float32)
    return g


def env_records(materials: list, n: int, n_sg: int, seed: int) -> np.ndarray:
    """Shading records over several materials ((N, levels, bins) tuples):
    uniform footprints with fractional levels, outgoing directions uniform on
    the upper hemisphere, SG lobe indices uniform."""
    u = uniform(seed, 19, 7 * n).reshape(n, 7)
    r = np.zeros(n, dtype=ENV_RECORD_DTYPE)
    m = np.minimum((u[:, 0] * len(materials)).astype(np.int64), len(materials) - 1)
    Ns = np.array([mt[0] for mt in materials])[m]
    Ls = np.array([mt[1] for mt in materials])[m]
    r["x"] = np.minimum((u[:, 1] * Ns).astype(np.int64), Ns - 1)
    r["y"] = np.minimum((u[:, 2] * Ns).astype(np.int64), Ns - 1)
    r["level"] = (u[:, 3] * (Ls - 1)).astype(np.float32)
    r["wo"] = _hemisphere(u[:, 4], u[:, 5]).astype(np.float32)
    r["sg"] = np.minimum((u[:, 6] * n_sg).astype(np.int64), n_sg - 1)
    r["material"] = m
    return r
