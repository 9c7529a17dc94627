"""Pins of the clustered-layout oracle (Sec. 4.2 blocks and regions, Sec. 4.4
block-splitting range queries) against facts outside its own code: a
brute-force regrouping of the blocks, the density normalisation of an exactly
rank-one map, the point query of Eq. 4, the mean-of-points identity of Fig.
rangeAndPoint, and the area-weighted split of a range at a block border."""
import numpy as np
import pytest

import synth
from oracle import clustered as ocl
from oracle import ndf


def _hist(N, L, B, seed, kind="flakes"):
    m = synth.flake_map(N, max(4, N * N // 32), 0.3, seed) if kind == "flakes" else \
        synth.brushed_map(N, 0.05, 0.3, 4, seed)
    s, t = ndf.bin_index(m, B)
    return [ndf.level_histograms(s, t, l, B) for l in range(L)]


def _random_factors(lay, R, seed, signed=False):
    fac = {}
    for j, mem in enumerate(lay["members"]):
        if not mem:
            continue
        u = synth.uniform(seed, j, (2 * lay["t"] + len(mem) + 1) * R)
        if signed:
            u = 2 * u - 1
        t = lay["t"]
        X = u[:t * R].reshape(t, R)
        Y = u[t * R:2 * t * R].reshape(t, R)
        Z = u[2 * t * R:(2 * t + len(mem)) * R].reshape(len(mem), R)
        lam = 0.5 + u[-R:]
        fac[j] = (lam, X, Y, Z, [])
    return fac


def test_layout_against_brute_force_regrouping():
    N, L, B = 16, 5, 32
    H = _hist(N, L, B, 3)
    lay = ocl.layout(H, B)
    t, nb = lay["t"], lay["nb"]
    assert (t, nb, lay["G"]) == (16, 2, 4 * 4)
    seen = 0
    for l in range(L):
        for y in range(N):
            for x in range(N):
                for bs in range(nb):
                    for bt in range(nb):
                        blk = H[l][y, x, bs * t:(bs + 1) * t, bt * t:(bt + 1) * t]
                        z = lay["zmap"][l, y, x, bs * nb + bt]
                        j = (((y // 8) * (N // 8) + x // 8) * nb + bs) * nb + bt
                        if blk.sum() == 0:
                            assert z == -1
                        else:
                            assert lay["members"][j][z] == (l, y, x)
                            seen += 1
    assert seen == sum(len(m) for m in lay["members"])
    for j, mem in enumerate(lay["members"]):
        assert mem == sorted(mem)  # level, then y, then x
        D = ocl.group_tensor(H, lay, j, raw_counts=True)
        assert D.shape[2] == len(mem) and (len(mem) == 0 or np.all(D.reshape(-1, len(mem)).sum(0) > 0))


def test_constant_map_is_rank_one_and_integrates_to_one():
    # every texel in bin (5, 20): every footprint's image is 4^l at that bin,
    # so each non-empty group is exactly rank one and the density's mean over
    # the whole [-1, 1]^2 image is 1/4
    N, L, B = 16, 5, 32
    s = np.full((N, N), 5)
    t = np.full((N, N), 20)
    H = [ndf.level_histograms(s, t, l, B) for l in range(L)]
    lay = ocl.layout(H, B)
    nonempty = [j for j, m in enumerate(lay["members"]) if m]
    assert len(nonempty) == (N // 8) ** 2  # one block position per region
    init = {j: [synth.uniform(9, 3 * j + k, n).reshape(n, 1) for k, n in
                enumerate((lay["t"], lay["t"], len(lay["members"][j])))] for j in nonempty}
    fac = ocl.decompose(H, lay, 1, init, sweeps=2)
    for j in nonempty:
        assert fac[j][4][-1] >= 1 - 1e-12
    q = np.zeros(3, dtype=synth.QUERY_DTYPE)
    q["x"], q["y"], q["level"] = [3, 9, 15], [0, 7, 12], [0.0, 2.5, 4.0]
    q["s0"], q["s1"], q["t0"], q["t1"] = 0.0, float(B), 0.0, float(B)
    assert np.allclose(ocl.range_query(lay, fac, q), 0.25, rtol=1e-12)
    q["s0"], q["s1"], q["t0"], q["t1"] = 5.0, 6.0, 20.0, 21.0
    assert np.allclose(ocl.range_query(lay, fac, q), B * B / 4.0, rtol=1e-12)


def test_point_mean_of_points_and_block_split():
    N, L, B, R = 16, 5, 32, 3
    H = _hist(N, L, B, 11, "brushed")
    lay = ocl.layout(H, B)
    fac = _random_factors(lay, R, 5, signed=True)
    img = ocl.reconstruct_image(lay, fac, 2, 9, 4)
    q = np.zeros(1, dtype=synth.QUERY_DTYPE)
    q["x"], q["y"], q["level"] = 4, 9, 2.0
    # Eq. 4: a zero-width range is the point value
    q["s0"] = q["s1"] = 13.5
    q["t0"] = q["t1"] = 17.0
    assert ocl.range_query(lay, fac, q)[0] == pytest.approx(img[13, 17], rel=1e-12)
    # Fig. rangeAndPoint: an integer range is the mean of its point values
    q["s0"], q["s1"], q["t0"], q["t1"] = 12.0, 19.0, 14.0, 18.0
    assert ocl.range_query(lay, fac, q)[0] == pytest.approx(img[12:19, 14:18].mean(), rel=1e-12)
    # a range across the block border s = 16 is the area-weighted sum of its parts
    q["s0"], q["s1"], q["t0"], q["t1"] = 10.25, 21.5, 3.75, 9.0
    whole = ocl.range_query(lay, fac, q)[0]
    a = q.copy(); a["s1"] = 16.0
    b = q.copy(); b["s0"] = 16.0
    wa, wb = (16.0 - 10.25) / (21.5 - 10.25), (21.5 - 16.0) / (21.5 - 10.25)
    assert whole == pytest.approx(wa * ocl.range_query(lay, fac, a)[0] + wb * ocl.range_query(lay, fac, b)[0],
                                  rel=1e-12)
    # blank blocks read 0; fractional levels blend linearly
    q["level"] = 2.25
    q2 = q.copy(); q2["level"] = 3.0
    q0 = q.copy(); q0["level"] = 2.0
    assert ocl.range_query(lay, fac, q)[0] == pytest.approx(
        0.75 * ocl.range_query(lay, fac, q0)[0] + 0.25 * ocl.range_query(lay, fac, q2)[0], rel=1e-12)


def test_compression_drops_blank_blocks():
    N, L, B = 16, 5, 64  # 16 x 16 blocks of a 64 x 64 image: 16 block positions
    H = _hist(N, L, B, 2)
    lay = ocl.layout(H, B)
    kept = sum(len(m) for m in lay["members"])
    total = L * N * N * lay["nb"] ** 2
    assert 0 < kept < total / 2  # concentrated normals: most blocks are blank
    r16 = ocl.compression_ratio(lay, 16)
    assert r16 == pytest.approx(
        sum(16 * (2 * 16 + len(m) + 1) + 2 * 16 * 17 for m in lay["members"] if m) / (L * N * N * B * B))
