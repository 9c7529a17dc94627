"""Pins of the structured MTTKRP oracle (O7b: the window moved from the
footprint tensor onto the spatial factors) and of the chunked sum of squares
against the definitions: the dense MTTKRP of the brute-force histogram tensor
(Sec. 4.1 counted texel by texel), closed forms of the norm at the finest and
coarsest levels, and CP-ALS on the dense tensor."""
import numpy as np
import pytest

import synth
from oracle import cp, ndf


def _maps(N, B, seed, kind):
    m = synth.flake_map(N, max(4, N * N // 16), 0.4, seed) if kind == "flakes" else \
        synth.brushed_map(N, 0.05, 0.3, 3, seed)
    return ndf.bin_index(m, B)


@pytest.mark.parametrize("N,L,B,R,kind", [(8, 4, 4, 3, "flakes"), (16, 5, 8, 2, "brushed"),
                                          (16, 3, 4, 5, "flakes"), (4, 3, 4, 1, "flakes")])
@pytest.mark.parametrize("raw", [False, True])
def test_structured_mttkrp_equals_dense_definition(N, L, B, R, kind, raw):
    s, t = _maps(N, B, 11 + N + L, kind)
    H = ndf.footprint_histograms_brute(s, t, L, B)
    X = ndf.logical(H.astype(np.float64) if raw else ndf.normalised_tensor(H, B))
    SF = cp.StructuredFootprint(s, t, L, B, raw_counts=raw)
    A = [2 * synth.uniform(19, k, n * R).reshape(n, R) - 1 for k, n in enumerate(X.shape)]
    for n in range(5):
        ref = cp.mttkrp_dense(X, A, n)
        got = SF.mttkrp(A, n)
        assert got.shape == ref.shape
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) <= 1e-12 * scale, n


def test_window_tables_hand_worked():
    # N = 4, level 1: w = 2, a = 1; alpha(u) = f[u + 1] + f[u] (mod 4) and the
    # footprint window of x covers x - 1, x
    SF = cp.StructuredFootprint(np.zeros((4, 4), int), np.zeros((4, 4), int), 3, 4)
    f = np.array([[1.0], [10.0], [100.0], [1000.0]])
    assert SF.window_adjoint(f, 1)[:, 0].tolist() == [11.0, 110.0, 1100.0, 1001.0]
    assert SF.window(f, 1)[:, 0].tolist() == [1001.0, 11.0, 110.0, 1100.0]
    # level 2 covers the whole map
    assert SF.window_adjoint(f, 2)[:, 0].tolist() == [1111.0] * 4


@pytest.mark.parametrize("N,L,B", [(8, 4, 4), (16, 5, 8)])
def test_level_sumsq_equals_definition(N, L, B):
    s, t = _maps(N, B, 5 + N, "flakes")
    H = ndf.footprint_histograms_brute(s, t, L, B)
    for l in range(L):
        assert ndf.level_sumsq(s, t, l, B, chunk=3) == int(np.sum(H[l] ** 2))
    # level 0: one texel per footprint; the whole map: every footprint holds
    # the map's own histogram
    n_b = np.bincount((s * B + t).ravel(), minlength=B * B)
    assert ndf.level_sumsq(s, t, 0, B) == N * N
    assert ndf.level_sumsq(s, t, L - 1, B) == N * N * int(np.sum(n_b ** 2))


def test_structured_als_equals_dense_als():
    N, L, B, R = 8, 4, 8, 4
    s, t = _maps(N, B, 3, "brushed")
    H = ndf.footprint_histograms_brute(s, t, L, B)
    X = ndf.logical(ndf.normalised_tensor(H, B))
    SF = cp.StructuredFootprint(s, t, L, B)
    assert abs(SF.norm2() - np.sum(X ** 2)) <= 1e-12 * np.sum(X ** 2)
    init = [synth.uniform(23, k, n * R).reshape(n, R) for k, n in enumerate(X.shape)]
    l1, A1, f1 = cp.cp_als(X, R, init, sweeps=4)
    l2, A2, f2 = cp.cp_als(SF, R, init, sweeps=4, fit_method="gram")
    assert np.allclose(f1, f2, rtol=0, atol=1e-9)
    assert np.allclose(l1, l2, rtol=1e-10, atol=0)
    for a, b in zip(A1, A2):
        assert np.allclose(a, b, rtol=0, atol=1e-10)
    with pytest.raises(ValueError):
        cp.cp_als(SF, R, init, sweeps=1)


def _gaussian_dense(s, t, L, B):
    H = np.stack([ndf.gaussian_histograms(s, t, l, B) for l in range(L)])  # [l][y][x][s][t]
    return np.transpose(H, (2, 1, 0, 3, 4)) * (B * B / 4.0)


def test_gaussian_weights():
    # normalised, symmetric, the support and sigma of the reading
    for N, l in ((16, 0), (16, 2), (16, 4), (1024, 10), (1024, 3)):
        g = ndf.gaussian_weights(l, N)
        rho = ndf.gaussian_radius(l, N)
        assert abs(g.sum() - 1.0) < 1e-15
        assert np.allclose(g, g[(-np.arange(N)) % N], rtol=0, atol=0)
        assert np.count_nonzero(g) == 2 * rho + 1
        sig = ndf.gaussian_sigma(l)
        assert sig == pytest.approx(1.5 * 2 ** l / np.sqrt(12.0))
        if rho >= 2:  # the ratio of neighbouring weights fixes sigma
            assert g[1] / g[0] == pytest.approx(np.exp(-1 / (2 * sig * sig)), rel=1e-12)
    assert ndf.gaussian_radius(0, 64) == 2 and ndf.gaussian_radius(10, 1024) == 511


@pytest.mark.parametrize("N,L,B,R", [(8, 4, 4, 3), (16, 5, 4, 2)])
def test_gaussian_structured_mttkrp_equals_dense_definition(N, L, B, R):
    s, t = _maps(N, B, 31 + N, "flakes")
    X = _gaussian_dense(s, t, L, B)
    SF = cp.StructuredFootprint(s, t, L, B, footprint="gaussian")
    A = [2 * synth.uniform(29, k, n * R).reshape(n, R) - 1 for k, n in enumerate(X.shape)]
    for n in range(5):
        ref = cp.mttkrp_dense(X, A, n)
        assert np.max(np.abs(SF.mttkrp(A, n) - ref)) <= 1e-12 * np.max(np.abs(ref)), n
    # every footprint's weights sum to 1: the density integrates to 1 over [-1, 1]^2
    assert np.allclose(X.sum(axis=(3, 4)) * 4.0 / (B * B), 1.0, rtol=1e-13)


@pytest.mark.parametrize("N,L,B", [(8, 4, 4), (16, 5, 8)])
def test_gaussian_sumsq_equals_definition(N, L, B):
    s, t = _maps(N, B, 41 + N, "brushed")
    A = ndf.match_autocorrelation(s, t, B)
    assert A[0, 0] == N * N and A.sum() == int(np.sum(np.bincount((s * B + t).ravel()) ** 2))
    for l in range(L):
        H = ndf.gaussian_histograms(s, t, l, B)
        assert abs(ndf.gaussian_sumsq(A, l) - np.sum(H * H)) <= 1e-12 * np.sum(H * H)


def test_gaussian_structured_als_equals_dense_als():
    N, L, B, R = 8, 4, 4, 3
    s, t = _maps(N, B, 5, "flakes")
    X = _gaussian_dense(s, t, L, B)
    SF = cp.StructuredFootprint(s, t, L, B, footprint="gaussian")
    assert abs(SF.norm2() - np.sum(X ** 2)) <= 1e-12 * np.sum(X ** 2)
    init = [synth.uniform(37, k, n * R).reshape(n, R) for k, n in enumerate(X.shape)]
    _, _, f1 = cp.cp_als(X, R, init, sweeps=3)
    _, _, f2 = cp.cp_als(SF, R, init, sweeps=3, fit_method="gram")
    assert np.allclose(f1, f2, rtol=0, atol=1e-9)
