"""Oracle: hierarchical NDF importance sampling from range queries (test
infrastructure; imported only by tests, the smoke check and the bench's
CPU-baseline leg).

Sec. 5.2 (Fig. sampling): to sample a half-vector from the NDF image of a
footprint, start from the whole image, split it evenly into four quads, take
the four quads' average NDF values by range queries (Sec. 4.3), choose one quad
with probability proportional to its average, and repeat inside the chosen
quad until a single pixel (bin) remains; then perturb the sample uniformly
inside that bin.  Because the range query is exact, the probability of
reaching a bin is its NDF value divided by the image sum (Fig. sampleNDF).

Readings where the paper is silent (shared with the GPU kernel's contract):

* the image is the B x B bin grid of a footprint (x, y, level) of a CP
  material; a footprint is placed like a range query (x, y mod N, level
  clamped to [0, L-1] and blended linearly between floor(level) and the next);
* the paper first chooses one of its 16 x 16-pixel image blocks by their
  averages; with one global tensor there are no blocks, so the descent starts
  from the whole image (B a power of two);
* a CP approximation can be negative, so quad averages are clamped to 0 before
  they are used as probabilities; when all four are 0 the choice is uniform;
* the quads are taken in the order (s low, t low), (s low, t high),
  (s high, t low), (s high, t high), and quad k is chosen for the first k with
  u * total < (p_0 + ... + p_k), one uniform u per step;
* the sample is (s_bin + u_s, t_bin + u_t) in bin units; its pmf is the
  product of the chosen steps' probabilities, its value the chosen bin's
  average (its NDF value).

The material is a dict of FP64 factors as in oracle.query: fx, fy, flw, fs, ft.
"""
from __future__ import annotations

import numpy as np


def footprint_weights(mat: dict, x: int, y: int, level: float) -> np.ndarray:
    """c_r = fx[x, r] fy[y, r] ((1 - f) flw[l0, r] + f flw[l1, r]) of one footprint."""
    N, L = mat["fx"].shape[0], mat["flw"].shape[0]
    lev = min(max(float(level), 0.0), L - 1.0)
    l0 = int(np.floor(lev))
    f = lev - l0
    l1 = min(l0 + 1, L - 1)
    lv = (1.0 - f) * mat["flw"][l0] + f * mat["flw"][l1]
    return mat["fx"][x % N] * mat["fy"][y % N] * lv


def quad_averages(mat: dict, c: np.ndarray, s0: int, t0: int, half: int) -> np.ndarray:
    """The four range averages (Sec. 4.3, integer-aligned ranges) of the square
    [s0, s0 + 2 half) x [t0, t0 + 2 half), in the order 00, 01, 10, 11
    (first digit: s half, second: t half)."""
    fs, ft = mat["fs"], mat["ft"]
    sa = fs[s0:s0 + half].mean(axis=0)
    sb = fs[s0 + half:s0 + 2 * half].mean(axis=0)
    ta = ft[t0:t0 + half].mean(axis=0)
    tb = ft[t0 + half:t0 + 2 * half].mean(axis=0)
    return np.array([np.sum(c * sa * ta), np.sum(c * sa * tb), np.sum(c * sb * ta), np.sum(c * sb * tb)])


def choose(q4: np.ndarray, u: float):
    """Clamp, then the first k with u * total < cumulative sum (uniform when all
    four are 0).  Returns (k, probability of k, margin) where margin is the
    distance of u * total to the nearest decision boundary, relative to total
    (how far the choice is from flipping)."""
    p = np.maximum(q4, 0.0)
    tot = float(p.sum())
    if tot <= 0.0:
        k = min(3, int(u * 4.0))
        return k, 0.25, abs(u * 4.0 - round(u * 4.0)) / 4.0
    target = u * tot
    cum = np.cumsum(p)
    k = int(np.searchsorted(cum, target, side="right"))
    k = min(k, 3)
    while p[k] <= 0.0 and k > 0:  # never land on a zero quad
        k -= 1
    bounds = np.concatenate([[0.0], cum])
    margin = float(np.min(np.abs(bounds[1:4] - target))) / tot
    return k, float(p[k] / tot), margin


def sample(mat: dict, x: int, y: int, level: float, u: np.ndarray):
    """One hierarchical sample: returns (s, t, pmf, value, min_margin)."""
    B = mat["fs"].shape[0]
    steps = int(round(np.log2(B)))
    assert 1 << steps == B, "the descent needs a power-of-two bin count"
    c = footprint_weights(mat, x, y, level)
    s0 = t0 = 0
    size = B
    pmf, value, margin = 1.0, 0.0, np.inf
    for k in range(steps):
        half = size // 2
        q4 = quad_averages(mat, c, s0, t0, half)
        ch, p, m = choose(q4, float(u[k]))
        pmf *= p
        margin = min(margin, m)
        value = float(q4[ch])
        if ch >= 2:
            s0 += half
        if ch & 1:
            t0 += half
        size = half
    return s0 + float(u[6]), t0 + float(u[7]), pmf, value, margin


def sample_batch(materials, samples: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Every sample of a batch (structured array with x, y, level, material;
    u: [n][8]); returns [n][5]: s, t, pmf, value, margin."""
    if isinstance(materials, dict):
        materials = [materials]
    out = np.empty((len(samples), 5))
    for i, smp in enumerate(samples):
        out[i] = sample(materials[int(smp["material"])], int(smp["x"]), int(smp["y"]),
                        float(smp["level"]), u[i])
    return out


def bin_pmf(mat: dict, x: int, y: int, level: float) -> np.ndarray:
    """Probability of every bin under the descent, [B][B]: the product of the
    step probabilities along the path to the bin (every path enumerated)."""
    B = mat["fs"].shape[0]
    c = footprint_weights(mat, x, y, level)
    out = np.zeros((B, B))

    def rec(s0, t0, size, prob):
        if size == 1:
            out[s0, t0] = prob
            return
        half = size // 2
        p = np.maximum(quad_averages(mat, c, s0, t0, half), 0.0)
        tot = p.sum()
        p = p / tot if tot > 0 else np.full(4, 0.25)
        for k in range(4):
            rec(s0 + (half if k >= 2 else 0), t0 + (half if k & 1 else 0), half, prob * p[k])

    rec(0, 0, B, 1.0)
    return out


def ndf_image(mat: dict, x: int, y: int, level: float) -> np.ndarray:
    """The footprint's NDF image, [B][B]: sum_r c_r fs[s, r] ft[t, r] (point
    queries of Eq. 4 for every bin)."""
    c = footprint_weights(mat, x, y, level)
    return np.einsum("r,sr,tr->st", c, mat["fs"], mat["ft"])
