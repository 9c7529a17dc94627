"""Pins for the oracle's CP-ALS (Sec. 4.2, Eq. 3; Kolda & Bader CP-ALS)."""
import numpy as np
import pytest

import synth
from oracle import cp, ndf


def _planted(shape, R, seed, cond=True):
    fac = []
    for m, n in enumerate(shape):
        u = synth.uniform(seed, 30 + m, n * R).reshape(n, R)
        A = u + (0.5 if cond else 0.0)
        if cond and n >= R:
            # well-conditioned columns: orthonormalise, then mix a little
            Q, _ = np.linalg.qr(2 * u - 1)
            A = Q[:, :R] + 0.2 * (u - 0.5)
        elif cond:
            # more ranks than rows: generic signed columns (Kruskal's uniqueness
            # condition still holds through the other modes)
            A = 2 * u - 1
        fac.append(A)
    lam = 1.0 + np.arange(R, dtype=np.float64)
    return lam, fac


def test_mttkrp_matches_loops():
    shape, R = (3, 4, 2, 3, 2), 2
    X = synth.uniform(1, 1, int(np.prod(shape))).reshape(shape)
    A = [synth.uniform(2, m, n * R).reshape(n, R) for m, n in enumerate(shape)]
    for n in range(5):
        M = cp.mttkrp_dense(X, A, n)
        ref = np.zeros((shape[n], R))
        for idx in np.ndindex(*shape):
            prod = np.ones(R)
            for m in range(5):
                if m != n:
                    prod = prod * A[m][idx[m]]
            ref[idx[n]] += X[idx] * prod
        assert np.allclose(M, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("R", [3, 5, 8])
def test_planted_low_rank_recovery(R):
    shape = (12, 10, 6, 8, 8)
    lam, fac = _planted(shape, R, 100 + R)
    X = cp.reconstruct(lam, fac)
    # the planted factors have mixed signs, so start from signed U[-1, 1)
    init = [2 * synth.uniform(2000 + R, m, n * R).reshape(n, R) - 1 for m, n in enumerate(shape)]
    lam_h, A, fits = cp.cp_als(X, R, init, sweeps=2000, tol=1e-15)
    resid = np.linalg.norm((X - cp.reconstruct(lam_h, A)).ravel()) / np.linalg.norm(X.ravel())
    assert resid <= 1e-10
    # factor congruence up to permutation and sign (scale is in lambda)
    for m in range(5):
        Ft = fac[m] / np.linalg.norm(fac[m], axis=0)
        C = np.abs(Ft.T @ A[m])
        assert np.all(np.max(C, axis=1) >= 1 - 1e-8)


def test_matrix_special_case_is_truncated_svd():
    # three modes of size 1: CP-ALS reduces to a rank-R matrix approximation,
    # whose optimum is the truncated SVD (Eckart-Young)
    I, J, R = 30, 20, 4
    M = synth.uniform(5, 5, I * J).reshape(I, J)
    X = M.reshape(I, J, 1, 1, 1)
    init = [synth.uniform(6, m, n * R).reshape(n, R) for m, n in enumerate(X.shape)]
    _, _, fits = cp.cp_als(X, R, init, sweeps=500)
    sv = np.linalg.svd(M, compute_uv=False)
    best = 1.0 - np.sqrt(np.sum(sv[R:] ** 2)) / np.linalg.norm(M)
    assert abs(fits[-1] - best) < 1e-8


def test_fit_monotone_on_footprint_tensor():
    w = synth.WORKLOADS["flakes32"]
    s, t = ndf.bin_index(synth.make_map(w), w["bins"])
    H = ndf.footprint_histograms(s, t, w["levels"], w["bins"])
    X = ndf.logical(ndf.normalised_tensor(H, w["bins"]))
    R = w["rank"]
    f = synth.init_factors(w["N"], w["levels"], w["bins"], R, 2001)
    init = [f["fx"], f["fy"], f["fl"], f["fs"], f["ft"]]
    _, _, fits = cp.cp_als(X, R, init, sweeps=12)
    assert np.all(np.diff(fits) >= -1e-12)
    assert 0.0 < fits[-1] < 1.0


def test_rank_one_data_one_sweep():
    shape = (5, 4, 3, 6, 2)
    lam, fac = _planted(shape, 1, 9, cond=False)
    X = cp.reconstruct(lam, fac)
    init = [synth.uniform(4, m, n).reshape(n, 1) for m, n in enumerate(shape)]
    _, _, fits = cp.cp_als(X, 1, init, sweeps=1)
    assert fits[0] >= 1 - 1e-12


def test_footprint_tensor_streaming_equals_dense():
    N, L, B, R = 8, 4, 4, 3
    m = synth.flake_map(N, 10, 0.4, 3)
    s, t = ndf.bin_index(m, B)
    H = ndf.footprint_histograms(s, t, L, B)
    X = ndf.logical(ndf.normalised_tensor(H, B))
    FT = cp.FootprintTensor(H, B)
    assert np.allclose(FT.dense_logical(), X, rtol=0, atol=0)
    A = [synth.uniform(7, k, n * R).reshape(n, R) for k, n in enumerate(X.shape)]
    for n in range(5):
        assert np.allclose(FT.mttkrp(A, n), cp.mttkrp_dense(X, A, n), rtol=1e-12, atol=0)
    lam = np.array([1.0, 2.0, 0.5])
    assert abs(FT.fit(lam, A) - cp.fit_dense(X, lam, A)) < 1e-12
    assert abs(FT.norm2() - np.sum(X ** 2)) <= 1e-12 * np.sum(X ** 2)
    init = [a.copy() for a in A]
    l1, A1, f1 = cp.cp_als(X, R, init, sweeps=3)
    l2, A2, f2 = cp.cp_als(FT, R, init, sweeps=3)
    assert np.allclose(f1, f2, rtol=0, atol=1e-12)


def test_to_material_folds_weights():
    lam = np.array([2.0, 3.0])
    fac = [np.ones((2, 2)), np.ones((2, 2)), np.array([[1.0, 1.0], [0.5, 2.0]]), np.ones((3, 2)), np.ones((3, 2))]
    m = cp.to_material(lam, fac)
    assert np.array_equal(m["flw"], np.array([[2.0, 3.0], [1.0, 6.0]]))


def test_gram_fit_equals_explicit_fit():
    w = synth.WORKLOADS["flakes32"]
    s, t = ndf.bin_index(synth.make_map(w), w["bins"])
    H = ndf.footprint_histograms(s, t, w["levels"], w["bins"])
    X = ndf.logical(ndf.normalised_tensor(H, w["bins"]))
    f = synth.init_factors(w["N"], w["levels"], w["bins"], 6, 2001)
    init = [f[k][:, :6] for k in ("fx", "fy", "fl", "fs", "ft")]
    _, _, fe = cp.cp_als(X, 6, init, sweeps=5)
    _, _, fg = cp.cp_als(X, 6, init, sweeps=5, fit_method="gram")
    FT = cp.FootprintTensor(H, w["bins"])
    _, _, ff = cp.cp_als(FT, 6, init, sweeps=5, fit_method="gram")
    assert np.allclose(fe, fg, rtol=0, atol=1e-9)
    assert np.allclose(fe, ff, rtol=0, atol=1e-9)
