"""Pins for the oracle's binning and footprint histograms (Sec. 4.1, Sec. 5.2)."""
import numpy as np
import pytest

import synth
from oracle import ndf


def test_bin_edges_hand_built():
    B = 8
    # values on bin edges go to the upper bin; -1 -> 0; +1 is clamped to B-1; -0.0 -> B/2
    nx = np.array([-1.0, -0.75, -0.5, -0.0, 0.0, 0.25, 0.999, 1.0, -0.76], dtype=np.float32)
    nxy = np.stack([nx, nx[::-1]], axis=-1)
    s, t = ndf.bin_index(nxy, B)
    assert s.tolist() == [0, 1, 2, 4, 4, 5, 7, 7, 0]
    assert t.tolist() == s[::-1].tolist()


def test_bin_fp32_rounding_not_fp64():
    # -1 + 2^-25 rounds to -1 in FP32, so (n.x + 1) is 0 in FP32 (bin 0) even
    # though the exact value is positive; the reading fixes FP32 evaluation.
    v = np.float32(-1.0 + 2.0 ** -24)  # representable
    s, _ = ndf.bin_index(np.array([[v, 0.0]], dtype=np.float32), 16)
    assert s[0] == 0
    # just below an interior edge in FP32 stays in the lower bin
    e = np.nextafter(np.float32(-0.5), np.float32(-1.0))
    s, _ = ndf.bin_index(np.array([[e, 0.0]], dtype=np.float32), 4)
    assert s[0] == 0
    s, _ = ndf.bin_index(np.array([[np.float32(-0.5), 0.0]], dtype=np.float32), 4)
    assert s[0] == 1


def test_nonfinite_rejected():
    with pytest.raises(ValueError):
        ndf.bin_index(np.array([[np.nan, 0.0]], dtype=np.float32), 4)
    with pytest.raises(ValueError):
        ndf.bin_index(np.array([[0.0, np.inf]], dtype=np.float32), 4)


def _random_bins(N, B, seed):
    u = synth.uniform(seed, 99, 2 * N * N)
    s = np.minimum((u[0::2] * B).astype(np.int64), B - 1).reshape(N, N)
    t = np.minimum((u[1::2] * B).astype(np.int64), B - 1).reshape(N, N)
    return s, t


@pytest.mark.parametrize("N,levels,B,seed", [(4, 3, 2, 1), (8, 4, 4, 2), (16, 5, 4, 3)])
def test_separable_equals_brute_force(N, levels, B, seed):
    s, t = _random_bins(N, B, seed)
    Hb = ndf.footprint_histograms_brute(s, t, levels, B)
    Hf = ndf.footprint_histograms(s, t, levels, B)
    assert np.array_equal(Hb, Hf)


def test_brute_force_on_flake_map():
    m = synth.flake_map(8, 6, 0.4, 5)
    s, t = ndf.bin_index(m, 4)
    assert np.array_equal(ndf.footprint_histograms_brute(s, t, 4, 4),
                          ndf.footprint_histograms(s, t, 4, 4))


def test_histogram_invariants_flakes32():
    w = synth.WORKLOADS["flakes32"]
    s, t = ndf.bin_index(synth.make_map(w), w["bins"])
    N, L1, B = w["N"], w["levels"], w["bins"]
    H = ndf.footprint_histograms(s, t, L1, B)
    # (1) every footprint holds 4^l texels
    for l in range(L1):
        assert np.all(H[l].sum(axis=(2, 3)) == 4 ** l)
    # (2) level 0 is one-hot at the texel's own bin
    yy, xx = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    assert np.all(H[0][yy, xx, s, t] == 1)
    assert H[0].sum() == N * N
    # (3) the top level (window = map) is the global histogram everywhere
    glob = np.bincount((s * B + t).ravel(), minlength=B * B).reshape(B, B)
    assert np.all(H[L1 - 1] == glob[None, None])
    # (4) doubling: W_{l+1}(x) = W_l(x - d) u W_l(x + d), d = 2^(l-1); W_1 = W_0(x-1) u W_0(x)
    for l in range(L1 - 1):
        lo, hi = (-1, 0) if l == 0 else (-(1 << (l - 1)), 1 << (l - 1))
        acc = np.zeros_like(H[l])
        for dy in (lo, hi):
            for dx in (lo, hi):
                acc += np.roll(np.roll(H[l], -dy, axis=0), -dx, axis=1)
        assert np.array_equal(acc, H[l + 1])
    # (5) window_histogram counts the same thing one footprint at a time
    for (x, y, l) in [(0, 0, 0), (5, 31, 3), (31, 7, 5), (17, 2, 4)]:
        assert np.array_equal(ndf.window_histogram(s, t, B, x, y, l), H[l, y, x])


def test_density_normalisation():
    # each NDF image integrates to one over [-1,1]^2 (bin area (2/B)^2)
    s, t = _random_bins(16, 8, 7)
    H = ndf.footprint_histograms(s, t, 5, 8)
    T = ndf.normalised_tensor(H, 8)
    integral = T.sum(axis=(3, 4)) * (2.0 / 8) ** 2
    assert np.allclose(integral, 1.0, rtol=0, atol=1e-15)


def test_window_centring():
    # a single marked texel appears, at level l, in exactly the footprints whose
    # window [x - a_l, x - a_l + 2^l) contains it
    N, B = 8, 2
    s = np.zeros((N, N), dtype=np.int64)
    t = np.zeros((N, N), dtype=np.int64)
    s[3, 5] = 1  # texel (x=5, y=3)
    H = ndf.footprint_histograms(s, t, 4, B)
    for l in range(4):
        w, a = 1 << l, ndf.window_offset(l)
        want = np.zeros((N, N), dtype=np.int64)
        for y in range(N):
            for x in range(N):
                inx = ((5 - (x - a)) % N) < w
                iny = ((3 - (y - a)) % N) < w
                want[y, x] = int(inx and iny)
        assert np.array_equal(H[l, :, :, 1, 0], want)
    assert ndf.window_offset(0) == 0 and ndf.window_offset(1) == 1 and ndf.window_offset(3) == 4
