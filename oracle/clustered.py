"""Oracle: the clustered compression layout of Sec. 4.2 (test infrastructure;
imported only by tests, the smoke check and the bench's CPU-baseline leg).

Sec. 4.2 does not decompose one global tensor.  It splits every NDF image
into t x t angular blocks (t = 16), groups the blocks of the footprints centred
in the same 8 x 8-texel region and lying at the same block position, stacks a
group's blocks into a t x t x M tensor (M = the number of blocks in the group),
drops the blocks that are completely blank, and decomposes every group by
CP-ALS (Eq. 3, one weight C_r and three vectors per rank).  A point query
(Eq. 4) reads one group; a range query (Eq. 5 with the 1D SATs of Sec. 4.4)
that crosses block borders is split at them.

Readings where the paper is silent (shared with the GPU kernels' contract):

* the footprints are this library's: a box footprint of every level at every
  texel (ndf.level_histograms), values T = H * B^2/(4*4^l) (or raw counts);
* t = min(16, B), B a multiple of t; regions are 8 x 8 texels (N >= 8), so the
  group of a footprint (x, y) is region (x // 8, y // 8) and block (s // t,
  t // t); a group stacks the footprints of every level in the order level,
  then y, then x, keeping the non-blank ones: z numbers the kept ones;
* the group's modes are (s', t', z) with s' = s - t*bs, t' = t - t*bt, and its
  CP-ALS is oracle.cp.cp_als with the mode order X (s'), Y (t'), Z (z), from
  given initial factors; a group with no member has no factors;
* a range query at a fractional level blends floor(level) and the next level
  linearly (clamped to [0, L-1]) like the global range query; its value is the
  average of the reconstructed, block-assembled NDF image over the bin
  rectangle [s0, s1] x [t0, t1] (ends clamped to [0, B], bin k = [k, k+1)),
  blank blocks reading 0; a zero-width range is the point value of the bin
  holding the end (B - 1 at B).
"""
from __future__ import annotations

import numpy as np

from . import cp, ndf


def block_size(bins: int) -> int:
    return min(16, bins)


def layout(H_levels, bins: int, region: int = 8) -> dict:
    """The clustered layout of count slices H_levels[l] ([N][N][B][B], [y][x][s][t]).
    Returns members (per group: list of (l, y, x)), zmap [L][N][N][nb*nb] (z or -1),
    and the dims.  Groups are numbered ((cy * (N / region) + cx) * nb + bs) * nb + bt."""
    L = len(H_levels)
    N = H_levels[0].shape[0]
    t = block_size(bins)
    nb = bins // t
    nr = N // region
    G = nr * nr * nb * nb
    members = [[] for _ in range(G)]
    zmap = np.full((L, N, N, nb * nb), -1, dtype=np.int64)
    for l in range(L):
        for y in range(N):
            for x in range(N):
                img = H_levels[l][y, x]
                for bs in range(nb):
                    for bt in range(nb):
                        blk = img[bs * t:(bs + 1) * t, bt * t:(bt + 1) * t]
                        if not np.any(blk):
                            continue
                        j = (((y // region) * nr + x // region) * nb + bs) * nb + bt
                        zmap[l, y, x, bs * nb + bt] = -2  # placeholder, numbered below
                        members[j].append((l, y, x))
    # z = position in the group's (level, y, x) order
    for j, mem in enumerate(members):
        mem.sort()
        bs, bt = (j // nb) % nb, j % nb
        for z, (l, y, x) in enumerate(mem):
            zmap[l, y, x, bs * nb + bt] = z
    return dict(N=N, L=L, B=bins, t=t, nb=nb, region=region, G=G, members=members, zmap=zmap)


def group_tensor(H_levels, lay: dict, j: int, raw_counts: bool = False) -> np.ndarray:
    """D_j[s'][t'][z] (FP64)."""
    t, nb, B = lay["t"], lay["nb"], lay["B"]
    bs, bt = (j // nb) % nb, j % nb
    mem = lay["members"][j]
    D = np.zeros((t, t, len(mem)))
    for z, (l, y, x) in enumerate(mem):
        sc = 1.0 if raw_counts else ndf.density_scale(l, B)
        D[:, :, z] = H_levels[l][y, x, bs * t:(bs + 1) * t, bt * t:(bt + 1) * t] * sc
    return D


def decompose(H_levels, lay: dict, rank: int, init: dict, sweeps: int, tol: float = 0.0,
              raw_counts: bool = False) -> dict:
    """CP-ALS of every non-empty group from init[j] = (X0, Y0, Z0).  Returns
    {j: (lam, X, Y, Z, fits)}."""
    out = {}
    for j, mem in enumerate(lay["members"]):
        if not mem:
            continue
        D = group_tensor(H_levels, lay, j, raw_counts)
        lam, A, fits = cp.cp_als(D, rank, list(init[j]), sweeps, tol)
        out[j] = (lam, A[0], A[1], A[2], fits)
    return out


def reconstruct_image(lay: dict, fac: dict, l: int, y: int, x: int) -> np.ndarray:
    """The block-assembled NDF image [B][B] of footprint (l, y, x) from the
    groups' CP factors; blank blocks are 0."""
    t, nb, B, region = lay["t"], lay["nb"], lay["B"], lay["region"]
    nr = lay["N"] // region
    img = np.zeros((B, B))
    for bs in range(nb):
        for bt in range(nb):
            z = lay["zmap"][l, y, x, bs * nb + bt]
            if z < 0:
                continue
            j = (((y // region) * nr + x // region) * nb + bs) * nb + bt
            lam, X, Y, Z, _ = fac[j]
            img[bs * t:(bs + 1) * t, bt * t:(bt + 1) * t] = np.einsum("r,sr,tr,r->st", lam, X, Y, Z[z])
    return img


def _axis_weights(a0: float, a1: float, B: int) -> np.ndarray:
    """Overlap of [a0, a1] with every bin [k, k+1), divided by the width; a
    zero width puts weight 1 on the bin holding a0 (B - 1 at B)."""
    a0, a1 = min(max(a0, 0.0), float(B)), min(max(a1, 0.0), float(B))
    if a1 < a0:
        a0, a1 = a1, a0
    w = np.zeros(B)
    if a1 == a0:
        w[min(int(np.floor(a0)), B - 1)] = 1.0
        return w
    for k in range(B):
        w[k] = max(0.0, min(a1, k + 1.0) - max(a0, float(k)))
    return w / (a1 - a0)


def range_query(lay: dict, fac: dict, queries: np.ndarray) -> np.ndarray:
    """Range average of every query (structured array x, y, level, s0, s1, t0, t1)
    over the reconstructed clustered tensor, FP64."""
    N, L, B = lay["N"], lay["L"], lay["B"]
    out = np.empty(len(queries))
    for i, q in enumerate(queries):
        x, y = int(q["x"]) % N, int(q["y"]) % N
        lev = min(max(float(q["level"]), 0.0), L - 1.0)
        l0 = int(np.floor(lev))
        f = lev - l0
        l1 = min(l0 + 1, L - 1)
        ws = _axis_weights(float(q["s0"]), float(q["s1"]), B)
        wt = _axis_weights(float(q["t0"]), float(q["t1"]), B)
        v0 = ws @ reconstruct_image(lay, fac, l0, y, x) @ wt
        v1 = ws @ reconstruct_image(lay, fac, l1, y, x) @ wt if f > 0 else 0.0
        out[i] = (1.0 - f) * v0 + f * v1
    return out


def compression_ratio(lay: dict, rank: int) -> float:
    """Stored floats (per group: X, Y, Z, the weights, and the two 1D SATs of
    X and Y, as Sec. 4.4 counts them) over the floats of the uncompressed tensor
    of all footprints."""
    t = lay["t"]
    stored = 0
    for mem in lay["members"]:
        if mem:
            stored += rank * (2 * t + len(mem) + 1) + 2 * rank * (t + 1)
    dense = lay["L"] * lay["N"] * lay["N"] * lay["B"] * lay["B"]
    return stored / dense
