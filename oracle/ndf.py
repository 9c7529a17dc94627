"""Oracle: normal binning and exhaustive footprint histograms (test infrastructure).

Sec. 4.1 precomputes one NDF image for every footprint of a multi-level
structure in which each level doubles the footprint size, until the footprint
covers the map.  This library's reading (the paper uses Gaussian-footprint
P-NDF images on a stride-32 grid; this path uses box footprints at every texel):

* an NDF image is the integer histogram of the projected normals (n.x, n.y) on a
  B x B grid over [-1, 1]^2 -- the "binning method" of Sec. 5.2 (Fig. 9 caption);
* level l has a 2^l x 2^l box footprint at every texel (x, y) of the tileable
  N x N map, with wraparound, l = 0 .. log2 N;
* the window is centred like the paper's footprints: W_l(x, y) covers texels
  ((x - a_l + i) mod N, (y - a_l + j) mod N), 0 <= i, j < 2^l, a_l = floor(2^l / 2).

Arrays are indexed [l][y][x][s][t]; the bin s comes from n.x and t from n.y.
"""
from __future__ import annotations

import numpy as np


def bin_index(nxy: np.ndarray, bins: int):
    """Bin (s, t) of every normal.  s = clamp(floor(fl32(fl32(n.x + 1) * fl32(B/2))),
    0, B-1), t likewise from n.y, evaluated in FP32 with round-to-nearest and no
    fused multiply-add.  A value on a bin edge belongs to the upper bin; n.x = 1
    is clamped into bin B-1.  Non-finite input raises ValueError."""
    nxy = np.asarray(nxy, dtype=np.float32)
    if not np.all(np.isfinite(nxy)):
        raise ValueError("non-finite normal")
    half = np.float32(bins / 2)
    one = np.float32(1.0)
    s = np.floor((nxy[..., 0] + one) * half)
    t = np.floor((nxy[..., 1] + one) * half)
    s = np.clip(s, 0, bins - 1).astype(np.int64)
    t = np.clip(t, 0, bins - 1).astype(np.int64)
    return s, t


def window_offset(level: int) -> int:
    """a_l = floor(2^l / 2): the footprint's offset from its corner to its centre."""
    return (1 << level) // 2


def footprint_histograms_brute(s: np.ndarray, t: np.ndarray, levels: int, bins: int) -> np.ndarray:
    """Definition written out with plain loops: for every level, texel and window
    texel, add one to the window's bin.  Tiny maps only."""
    N = s.shape[0]
    H = np.zeros((levels, N, N, bins, bins), dtype=np.int64)
    for l in range(levels):
        w, a = 1 << l, window_offset(l)
        for y in range(N):
            for x in range(N):
                for j in range(w):
                    for i in range(w):
                        u = (x - a + i) % N
                        v = (y - a + j) % N
                        H[l, y, x, s[v, u], t[v, u]] += 1
    return H


def _cyclic_window_sum(A: np.ndarray, axis: int, w: int, a: int) -> np.ndarray:
    """out[k] = sum_{i < w} A[(k - a + i) mod n] along `axis`, exact in int64.
    The sum is taken as a difference of running sums over two periods."""
    n = A.shape[axis]
    A2 = np.concatenate([A, A], axis=axis)
    C = np.cumsum(A2, axis=axis, dtype=np.int64)
    zero_shape = list(C.shape)
    zero_shape[axis] = 1
    C = np.concatenate([np.zeros(zero_shape, dtype=np.int64), C], axis=axis)
    start = (np.arange(n) - a) % n
    return np.take(C, start + w, axis=axis) - np.take(C, start, axis=axis)


def level_histograms(s: np.ndarray, t: np.ndarray, level: int, bins: int) -> np.ndarray:
    """H_l[y][x][s][t] for one level: the box window is separable, so the count
    is a window sum of the per-bin indicator along x followed by one along y."""
    N = s.shape[0]
    onehot = np.zeros((N, N, bins, bins), dtype=np.int64)
    yy, xx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    onehot[yy, xx, s, t] = 1
    w, a = 1 << level, window_offset(level)
    return _cyclic_window_sum(_cyclic_window_sum(onehot, 1, w, a), 0, w, a)


def level_sumsq(s: np.ndarray, t: np.ndarray, level: int, bins: int, chunk: int = 32) -> int:
    """Sum over every footprint (x, y) and bin of H_l[y][x][s][t]^2, exact.  The
    same separable window sums as level_histograms, taken over a few occupied
    bins at a time (a bin holding no texel has zero counts everywhere), so that
    the largest maps fit in host memory."""
    flat = s.astype(np.int64) * bins + t
    occupied = np.unique(flat)
    w, a = 1 << level, window_offset(level)
    total = 0
    for i in range(0, len(occupied), chunk):
        ids = occupied[i:i + chunk]
        onehot = (flat[:, :, None] == ids[None, None, :]).astype(np.int64)
        H = _cyclic_window_sum(_cyclic_window_sum(onehot, 1, w, a), 0, w, a)
        total += int(np.sum(H * H))
    return total


def footprint_histograms(s: np.ndarray, t: np.ndarray, levels: int, bins: int) -> np.ndarray:
    """All levels, int64 array [levels][y][x][s][t]."""
    N = s.shape[0]
    H = np.empty((levels, N, N, bins, bins), dtype=np.int64)
    for l in range(levels):
        H[l] = level_histograms(s, t, l, bins)
    return H


def window_histogram(s: np.ndarray, t: np.ndarray, bins: int, x: int, y: int, level: int) -> np.ndarray:
    """One footprint's histogram [B][B], counted directly from the texels of its
    window (used to check single outputs of full-size builds)."""
    N = s.shape[0]
    w, a = 1 << level, window_offset(level)
    xs = (x - a + np.arange(w)) % N
    ys = (y - a + np.arange(w)) % N
    flat = (s[np.ix_(ys, xs)] * bins + t[np.ix_(ys, xs)]).ravel()
    return np.bincount(flat, minlength=bins * bins).reshape(bins, bins)


def gaussian_sigma(level: int) -> float:
    """sigma_l = 1.5 * 2^l / sqrt(12): Sec. 4.1 sizes a footprint as a Gaussian of
    standard deviation 1.5 s / sqrt(12) for the sampling stride s; the box of
    level l (width 2^l) plays the stride here."""
    return 1.5 * float(1 << level) / np.sqrt(12.0)


def gaussian_radius(level: int, N: int) -> int:
    """Support half-width: ceil(3 sigma_l), at most floor((N - 1) / 2) so that
    the support never overlaps itself on the N-periodic map."""
    return int(min(np.ceil(3.0 * gaussian_sigma(level)), (N - 1) // 2))


def gaussian_weights(level: int, N: int) -> np.ndarray:
    """g_l[d mod N], d = -rho .. rho: exp(-d^2 / (2 sigma_l^2)) normalised to sum
    1 (Eq. geom's G_p, separable, truncated to the support); 0 elsewhere."""
    sig, rho = gaussian_sigma(level), gaussian_radius(level, N)
    d = np.arange(-rho, rho + 1)
    w = np.exp(-(d.astype(np.float64) ** 2) / (2.0 * sig * sig))
    g = np.zeros(N)
    g[d % N] = w / w.sum()
    return g


def gaussian_histograms(s: np.ndarray, t: np.ndarray, level: int, bins: int) -> np.ndarray:
    """Gaussian-footprint NDF weights of one level, [y][x][s][t] (FP64): the
    footprint of (x, y) weighs texel u by g_l(u_x - x) g_l(u_y - y).  Written
    out texel by texel: tiny maps only."""
    N = s.shape[0]
    g = gaussian_weights(level, N)
    H = np.zeros((N, N, bins, bins))
    for uy in range(N):
        for ux in range(N):
            wx = g[(ux - np.arange(N)) % N]  # over footprint centres x
            wy = g[(uy - np.arange(N)) % N]
            H[:, :, s[uy, ux], t[uy, ux]] += np.outer(wy, wx)
    return H


def match_autocorrelation(s: np.ndarray, t: np.ndarray, bins: int) -> np.ndarray:
    """A[e_y][e_x] = number of texels u whose bin equals the bin of u + e
    (cyclic), counted shift by shift."""
    b = s.astype(np.int64) * bins + t
    N = b.shape[0]
    A = np.zeros((N, N), dtype=np.int64)
    for ey in range(N):
        by = np.roll(b, -ey, axis=0)
        for ex in range(N):
            A[ey, ex] = int(np.count_nonzero(b == np.roll(by, -ex, axis=1)))
    return A


def gaussian_sumsq(A: np.ndarray, level: int) -> float:
    """Sum over footprints and bins of the squared Gaussian weights of one level,
    from the same-bin autocorrelation A: the sum over texel pairs (u, v) in a
    common bin of K(u_x - v_x) K(u_y - v_y), K(e) = sum_d g(d) g(d + e) being
    the number of ways a footprint weighs both (separable Gaussian)."""
    N = A.shape[0]
    g = gaussian_weights(level, N)
    K = np.array([np.dot(g, np.roll(g, -e)) for e in range(N)])
    return float(K @ A @ K)


def density_scale(level: int, bins: int) -> float:
    """Counts -> NDF values.  Eq. 2 normalises the footprint weight, so an NDF
    image is a density; over [-1,1]^2 with bin area (2/B)^2 the density of a bin
    holding c of the 4^l footprint texels is c * B^2 / (4 * 4^l)."""
    return bins * bins / (4.0 * float(4 ** level))


def normalised_tensor(H: np.ndarray, bins: int) -> np.ndarray:
    """T[l] = H[l] * B^2 / (4 * 4^l), FP64, same [l][y][x][s][t] order."""
    T = H.astype(np.float64)
    for l in range(H.shape[0]):
        T[l] *= density_scale(l, bins)
    return T


def logical(T_phys: np.ndarray) -> np.ndarray:
    """[l][y][x][s][t] -> logical mode order (x, y, l, s, t)."""
    return np.transpose(T_phys, (2, 1, 0, 3, 4))
