"""GPU parity of binning and footprint histograms (rows a1-a2): bit-exact."""
import numpy as np
import pytest
import torch

import synth
from oracle import ndf
from _gpu import dev, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def _bins_gpu(nxy, B):
    import paper_2109_14807_gb300 as g
    st = g.new_status()
    b = g.bin_normals(dev(nxy), B, status=st)
    return b.cpu().numpy().astype(np.int64) & 0xFFFF, g.status_bits(st)


def test_bins_bit_exact_maps_and_edges():
    for w in ("flakes32", "brushed512"):
        m = synth.make_map(synth.WORKLOADS[w])
        B = synth.WORKLOADS[w]["bins"]
        s, t = ndf.bin_index(m, B)
        code, st = _bins_gpu(m, B)
        assert st == 0
        assert np.array_equal(code, s * B + t)
    # values on and next to every bin edge, +-1, -0.0, and out-of-range finite values
    B = 16
    edges = np.float32(-1.0) + np.arange(B + 1, dtype=np.float32) * np.float32(2.0 / B)
    vals = np.concatenate([edges, np.nextafter(edges, np.float32(-2)), np.nextafter(edges, np.float32(2)),
                           np.array([-0.0, 0.0, 1.0, -1.0, 3.5, -7.0, 1e30, -1e30], np.float32)])
    n = int(np.ceil(np.sqrt(len(vals))))
    n = 1 << int(np.ceil(np.log2(n)))
    grid = np.zeros((n * n, 2), np.float32)
    grid[:len(vals), 0] = vals
    grid[:len(vals), 1] = vals[::-1]
    grid = grid.reshape(n, n, 2)
    s, t = ndf.bin_index(grid, B)
    code, st = _bins_gpu(grid, B)
    assert st == 0
    assert np.array_equal(code, s * B + t)


def test_nonfinite_normal_sets_status():
    m = synth.make_map(synth.WORKLOADS["flakes32"]).copy()
    m[3, 4, 0] = np.nan
    m[7, 1, 1] = np.inf
    _, st = _bins_gpu(m, 16)
    assert st & 0x1


def test_implicit_build_writes_the_bin_map():
    # a NULL histogram: the call writes only the bin map, of which every
    # footprint histogram is a box count (Sec. 4.1); the codes are the oracle's
    import paper_2109_14807_gb300 as g
    w = synth.WORKLOADS["flakes32"]
    m = synth.make_map(w).copy()
    B = w["bins"]
    s, t = ndf.bin_index(m, B)
    st = g.new_status()
    code = g.build_footprint_ndfs(dev(m), w["levels"], B, status=st, implicit=True)
    torch.cuda.synchronize()
    assert g.status_bits(st) == 0
    assert np.array_equal(code.cpu().numpy().astype(np.int64) & 0xFFFF, s * B + t)
    m[2, 5, 1] = np.nan
    st = g.new_status()
    g.build_footprint_ndfs(dev(m), w["levels"], B, status=st, implicit=True)
    assert g.status_bits(st) & 0x1


@pytest.mark.parametrize("N,L,B,kind", [(32, 6, 16, "flakes"), (64, 7, 32, "brushed"), (8, 4, 8, "flakes")])
def test_histograms_bit_exact_full(N, L, B, kind):
    import paper_2109_14807_gb300 as g
    if kind == "flakes":
        m = synth.flake_map(N, max(4, N * N // 16), 0.3, 11 + N)
    else:
        m = synth.brushed_map(N, 0.05, 0.3, 8, 12 + N)
    s, t = ndf.bin_index(m, B)
    ref = ndf.footprint_histograms(s, t, L, B)
    st = g.new_status()
    H = g.build_footprint_ndfs(dev(m), L, B, status=st)
    torch.cuda.synchronize()
    assert g.status_bits(st) == 0
    assert np.array_equal(H.cpu().numpy(), ref)


def _check_full_size(name, n_samples, seed):
    import paper_2109_14807_gb300 as g
    w = synth.WORKLOADS[name]
    N, L, B = w["N"], w["levels"], w["bins"]
    m = synth.make_map(w)
    s, t = ndf.bin_index(m, B)
    H = g.build_footprint_ndfs(dev(m), L, B)
    torch.cuda.synchronize()
    # invariant at every footprint: 4^l texels
    for l in range(L):
        sums = H[l].sum(dim=(2, 3), dtype=torch.int64)
        assert bool((sums == 4 ** l).all()), l
    # top level == global histogram everywhere
    glob = torch.from_numpy(np.bincount((s * B + t).ravel(), minlength=B * B).reshape(B, B)).cuda()
    assert bool((H[L - 1] == glob.to(torch.int32)).all())
    # sampled footprints counted one by one from their windows
    u = synth.uniform(seed, 1, 3 * n_samples)
    for i in range(n_samples):
        x = int(u[3 * i] * N)
        y = int(u[3 * i + 1] * N)
        l = i % L
        want = ndf.window_histogram(s, t, B, x, y, l)
        assert np.array_equal(H[l, y, x].cpu().numpy(), want), (x, y, l)
    del H
    torch.cuda.empty_cache()


def test_histograms_brushed512_sampled():
    _check_full_size("brushed512", 60, 5)


def test_histograms_flakes1024_sampled():
    _check_full_size("flakes1024", 44, 6)
