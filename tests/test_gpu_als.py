"""GPU parity of the CP-ALS path (rows a3-a4): the five MTTKRPs element by
element against the oracle's dense MTTKRP, and ALS fits against the FP64
oracle's CP-ALS from the same initial factors."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import cp, ndf
from _gpu import dev, lib, oracle_material, query_error, QUERY_TOL

pytestmark = pytest.mark.gpu

# MTTKRP tolerance relative to the magnitude scale sum |X| prod |A| of each entry:
# FP32 accumulation / TF32 (11-bit significand) / BF16 (8-bit significand) inputs
MTTKRP_TOL = {"fp32": 2e-5, "tf32": 3e-3, "bf16": 1.5e-2, "bf16_1x": 1.5e-2}
# ALS fit tolerance vs the FP64 oracle after the same sweeps from the same init.
# BF16 (tensor in BF16, Khatri-Rao operand as a BF16 hi + lo pair) must meet
# 1e-4.  Single-pass TF32 rounds the Khatri-Rao operand to 11 significant bits;
# emulating that rounding in FP64 on the 64^2 brushed workload gives ~9e-5 after
# 8 sweeps, so it is held to 2e-4.
FIT_TOL = {"bf16": 1e-4, "tf32": 2e-4}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def _tensor(N, L, B, kind, seed):
    m = synth.flake_map(N, max(4, N * N // 16), 0.3, seed) if kind == "flakes" else \
        synth.brushed_map(N, 0.05, 0.3, 6, seed)
    s, t = ndf.bin_index(m, B)
    H = ndf.footprint_histograms(s, t, L, B)
    return m, H, ndf.logical(ndf.normalised_tensor(H, B))


def _supported(prec, N, L, B, R):
    from paper_2109_14807_gb300 import _lib
    return _lib.load().gsp_cp_workspace_bytes(N, L, B, R, _lib.PREC[prec]) > 0


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16", "bf16_1x"])
@pytest.mark.parametrize("N,L,B,R", [(32, 6, 16, 8), (32, 6, 16, 16), (64, 7, 32, 32), (64, 7, 16, 64),
                                     (32, 6, 32, 64)])
def test_mttkrp_parity(prec, N, L, B, R):
    import paper_2109_14807_gb300 as g
    m, H, X = _tensor(N, L, B, "flakes", 20 + N + R)
    ws = g.CPWorkspace(N, L, B, R, prec) if _supported(prec, N, L, B, R) else None
    if ws is None:
        pytest.skip(f"{prec} MTTKRP does not support the shape {(N, L, B, R)}")
    ws.prepare(hist=dev(H, torch.int32))
    u = [synth.uniform(300 + R, k, n * R).reshape(n, R).astype(np.float32)
         for k, n in enumerate((N, N, L, B, B))]
    f = {k: dev(a) for k, a in zip(("fx", "fy", "fl", "fs", "ft"), u)}
    outs = ws.mttkrp(f)
    torch.cuda.synchronize()
    A = [a.astype(np.float64) for a in u]
    for n in range(5):
        ref = cp.mttkrp_dense(X, A, n)  # factors >= 0 and X >= 0: ref is its own scale
        got = outs[n].double().cpu().numpy()
        err = np.max(np.abs(got - ref) / np.maximum(ref, 1e-30 + np.max(ref) * 1e-6))
        assert err <= MTTKRP_TOL[prec], (n, err)


def _map_of_bins(N, B, bins, seed):
    """Normal map whose texels fall in the bins `bins` (cycled over the texels
    in a seeded random order), each normal at its bin's centre."""
    bins = np.asarray(bins)
    code = bins[np.arange(N * N) % len(bins)][np.argsort(synth.uniform(seed, 5, N * N))]
    s, t = code // B, code % B
    m = np.stack([(s + 0.5) / (B / 2) - 1.0, (t + 0.5) / (B / 2) - 1.0], axis=-1)
    return m.reshape(N, N, 2).astype(np.float32)


@pytest.mark.parametrize("prec", ["bf16", "fp32"])
@pytest.mark.parametrize("B,n_occ", [(8, 20), (16, 1), (16, 128), (16, 129), (16, 256), (32, 128),
                                     (32, 200), (32, 1024)])
def test_operand_columns_and_mttkrp_at_every_occupancy(prec, B, n_occ):
    # the operand keeps the bins that occur (increasing order), padded to a
    # multiple of 16 columns for the tensor-core precisions and of 128 for FP32
    # (all B^2 bins when B^2 < 256); the MTTKRPs are those of the full tensor
    # whatever the occupancy
    import paper_2109_14807_gb300 as g
    N, L, R = 64, 7, 16
    occ = np.sort(np.argsort(synth.uniform(40 + n_occ, B, B * B))[:n_occ])
    m = _map_of_bins(N, B, occ, 7 + n_occ)
    s, t = ndf.bin_index(m, B)
    assert np.array_equal(np.unique(s * B + t), occ)
    unit = 128 if prec == "fp32" else 16
    cols = B * B if B * B < 256 else min(B * B, max(unit, -(-n_occ // unit) * unit))
    if not _supported(prec, N, L, B, R):
        pytest.skip(f"{prec} MTTKRP does not support the shape {(N, L, B, R)}")
    ws = g.CPWorkspace(N, L, B, R, prec)
    ws.prepare(normal_xy=dev(m))
    assert ws.operand_cols() == ((B * B if B * B < 256 else n_occ), cols)
    H = ndf.footprint_histograms(s, t, L, B)
    X = ndf.logical(ndf.normalised_tensor(H, B))
    u = [synth.uniform(500 + B, k, n * R).reshape(n, R).astype(np.float32)
         for k, n in enumerate((N, N, L, B, B))]
    outs = ws.mttkrp({k: dev(a) for k, a in zip(("fx", "fy", "fl", "fs", "ft"), u)})
    torch.cuda.synchronize()
    A = [a.astype(np.float64) for a in u]
    for n in range(5):
        ref = cp.mttkrp_dense(X, A, n)
        got = outs[n].double().cpu().numpy()
        err = np.max(np.abs(got - ref) / np.maximum(ref, 1e-30 + np.max(ref) * 1e-6))
        assert err <= MTTKRP_TOL[prec], (n, err)
    # the same operand from the int32 histograms
    ws2 = g.CPWorkspace(N, L, B, R, prec)
    ws2.prepare(hist=dev(H, torch.int32))
    assert ws2.operand_cols() == ws.operand_cols()
    nb = L * N * N * cols * (2 if prec == "bf16" else 4)
    assert torch.equal(ws.operand_view(nb), ws2.operand_view(nb))


@pytest.mark.parametrize("n_occ", [200, 256])
def test_rank64_mttkrp_over_several_st_groups(n_occ):
    # rank 64 with the BF16 hi + lo pair: the Z' pass splits the stored
    # columns into groups of at most 80 (208 stored: 3 groups of 80, the last
    # reaching past the stored columns; 256: 4 groups of 64); all five MTTKRPs
    # against the dense oracle
    import paper_2109_14807_gb300 as g
    N, L, B, R = 64, 7, 16, 64
    if not _supported("bf16", N, L, B, R):
        pytest.skip(f"bf16 MTTKRP does not support the shape {(N, L, B, R)}")
    occ = np.sort(np.argsort(synth.uniform(60 + n_occ, B, B * B))[:n_occ])
    m = _map_of_bins(N, B, occ, 11 + n_occ)
    s, t = ndf.bin_index(m, B)
    assert np.array_equal(np.unique(s * B + t), occ)
    ws = g.CPWorkspace(N, L, B, R, "bf16")
    ws.prepare(normal_xy=dev(m))
    assert ws.operand_cols() == (n_occ, -(-n_occ // 16) * 16)
    X = ndf.logical(ndf.normalised_tensor(ndf.footprint_histograms(s, t, L, B), B))
    u = [synth.uniform(800 + n_occ, k, n * R).reshape(n, R).astype(np.float32)
         for k, n in enumerate((N, N, L, B, B))]
    outs = ws.mttkrp({k: dev(a) for k, a in zip(("fx", "fy", "fl", "fs", "ft"), u)})
    torch.cuda.synchronize()
    A = [a.astype(np.float64) for a in u]
    for n in range(5):
        ref = cp.mttkrp_dense(X, A, n)
        got = outs[n].double().cpu().numpy()
        err = np.max(np.abs(got - ref) / np.maximum(ref, 1e-30 + np.max(ref) * 1e-6))
        assert err <= MTTKRP_TOL["bf16"], (n, err)


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_operand_columns_at_128_bins(prec):
    # B = 128 (16384 bins, the largest bin grid): 300 bins occur, 384 operand
    # columns for FP32 (304 stored for TF32); the MTTKRPs against the
    # structured oracle (pinned to the dense definition), which never forms the
    # 16384-column tensor
    import paper_2109_14807_gb300 as g
    N, L, B, R = 64, 7, 128, 16
    if not _supported(prec, N, L, B, R):
        pytest.skip(f"{prec} MTTKRP does not support the shape {(N, L, B, R)}")
    occ = np.sort(np.argsort(synth.uniform(41, B, B * B))[:300])
    m = _map_of_bins(N, B, occ, 9)
    s, t = ndf.bin_index(m, B)
    ws = g.CPWorkspace(N, L, B, R, prec)
    ws.prepare(normal_xy=dev(m))
    assert ws.operand_cols() == (300, 384 if prec == "fp32" else 304)
    u = [synth.uniform(700, k, n * R).reshape(n, R).astype(np.float32) for k, n in enumerate((N, N, L, B, B))]
    outs = ws.mttkrp({k: dev(a) for k, a in zip(("fx", "fy", "fl", "fs", "ft"), u)})
    torch.cuda.synchronize()
    SF = cp.StructuredFootprint(s, t, L, B)
    A = [a.astype(np.float64) for a in u]
    for n in range(5):
        ref = SF.mttkrp(A, n)
        got = outs[n].double().cpu().numpy()
        err = np.max(np.abs(got - ref) / np.maximum(ref, 1e-30 + np.max(ref) * 1e-6))
        assert err <= MTTKRP_TOL[prec], (n, err)


def _oracle_fits(X, R, init, sweeps):
    A0 = [init[k].astype(np.float32).astype(np.float64) for k in ("fx", "fy", "fl", "fs", "ft")]
    return cp.cp_als(X, R, A0, sweeps)


def test_als_fp32_flakes32_matches_oracle():
    import paper_2109_14807_gb300 as g
    w = synth.WORKLOADS["flakes32"]
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    m = synth.make_map(w)
    s, t = ndf.bin_index(m, B)
    H = ndf.footprint_histograms(s, t, L, B)
    X = ndf.logical(ndf.normalised_tensor(H, B))
    init = synth.init_factors(N, L, B, R, 2001)
    _, _, ofits = _oracle_fits(X, R, init, w["sweeps"])
    f, fits, fb = g.cp_decompose(R, init, hist=dev(H, torch.int32), sweeps=w["sweeps"], precision="fp32")
    assert fb == 0
    fits = np.array(fits)
    rel = np.abs(fits - ofits) / np.abs(ofits)
    assert np.max(rel) <= 1e-5, (fits, ofits)
    # the same factors answer queries like the oracle does
    mat = g.QueryMaterial.from_factors(f)
    g.build_query_tables(mat)
    q = synth.queries_integer(N, L, B, w["queries"], 1001)
    got = g.range_query(mat, g.queries_to_device(q)).cpu().numpy()
    err, _ = query_error(got, oracle_material(f), q)
    assert err <= QUERY_TOL


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32"])
def test_als_from_normals_equals_from_histograms(prec):
    # both ways of preparing the operand give the same values (the rounding of
    # the tensor-core operands depends only on the element index)
    import paper_2109_14807_gb300 as g
    N, L, B, R = 64, 7, 16, 16
    if not _supported(prec, N, L, B, R):
        pytest.skip(f"{prec} path unavailable")
    m = synth.flake_map(N, 256, 0.15, 1)
    init = synth.init_factors(N, L, B, R, 2001)
    H = g.build_footprint_ndfs(dev(m), L, B)
    _, fits1, _ = g.cp_decompose(R, init, hist=H, sweeps=5, precision=prec)
    _, fits2, _ = g.cp_decompose(R, init, normal_xy=dev(m), levels=L, bins=B, sweeps=5,
                                 precision=prec)
    assert fits1 == fits2


@pytest.mark.parametrize("prec,drop", [("bf16", 16), ("tf32", 13)])
def test_operand_rounding_is_exact_or_neighbour_and_unbiased(prec, drop):
    # The tensor-core operand (documented as levels*N^2*columns elements from
    # the workspace's operand offset) holds every exactly representable density unchanged and
    # every other one as its lower or upper neighbour on the BF16 / TF32 grid,
    # without bias: the summed rounding error stays within six standard
    # deviations of a sum of independent zero-mean errors of at most one ulp.
    # 16 large flakes put thousands of texels of one bin in the coarse
    # footprints (counts above 256 and 2048 are not representable).
    import paper_2109_14807_gb300 as g
    N, L, B, R = 128, 8, 16, 16
    if not _supported(prec, N, L, B, R):
        pytest.skip(f"{prec} path unavailable")
    m = synth.flake_map(N, 16, 0.1, 77)
    s, t = ndf.bin_index(m, B)
    H = ndf.footprint_histograms(s, t, L, B)
    # operand columns: the bins occurring in the map, in increasing order, then
    # zero columns up to a multiple of 16 (the tensor-core precisions)
    occ = np.unique(s * B + t)
    Bk = min(B * B, max(16, -(-len(occ) // 16) * 16))
    dense = ndf.normalised_tensor(H, B).reshape(L, N, N, B * B)
    exact = np.zeros((L, N, N, Bk), dtype=np.float32)
    exact[..., :len(occ)] = dense[..., occ]  # exact: counts * 2^k
    exact = exact.ravel()
    del dense
    ws = g.CPWorkspace(N, L, B, R, prec)
    ws.prepare(normal_xy=dev(m))
    torch.cuda.synchronize()
    assert ws.operand_cols() == (len(occ), Bk)
    n = exact.size
    if prec == "bf16":
        raw = ws.operand_view(2 * n).cpu().numpy().view(np.uint16).astype(np.uint64) << 16
    else:
        raw = ws.operand_view(4 * n).cpu().numpy().view(np.uint32).astype(np.uint64)
    u = exact.view(np.uint32).astype(np.uint64)
    lo = (u >> drop) << drop
    up = lo + (1 << drop)
    representable = lo == u
    assert np.all(raw[representable] == u[representable])
    assert np.all((raw == lo) | (raw == up))
    f = lambda b: b.astype(np.uint32).view(np.float32).astype(np.float64)
    err = f(raw) - exact.astype(np.float64)
    ulp = f(up) - f(lo)
    inexact = ~representable
    assert np.count_nonzero(inexact) > 10_000  # the case exercises the rounding
    del H
    bound = 6.0 * np.sqrt(np.sum(ulp[inexact] ** 2) / 4.0)
    assert abs(np.sum(err)) <= bound, (np.sum(err), bound)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_als_tensor_core_fit_matches_oracle_mid(prec):
    import paper_2109_14807_gb300 as g
    N, L, B, R = 64, 7, 32, 32
    if not _supported(prec, N, L, B, R):
        pytest.skip(f"{prec} path unavailable")
    m, H, X = _tensor(N, L, B, "brushed", 77)
    init = synth.init_factors(N, L, B, R, 2077)
    sweeps = 8
    _, _, ofits = _oracle_fits(X, R, init, sweeps)
    _, fits, _ = g.cp_decompose(R, init, hist=dev(H, torch.int32), sweeps=sweeps, precision=prec)
    rel = np.abs(np.array(fits) - ofits) / np.abs(ofits)
    assert np.max(rel) <= FIT_TOL[prec], (fits, ofits)


def test_als_resume_is_bit_identical():
    import paper_2109_14807_gb300 as g
    w = synth.WORKLOADS["flakes32"]
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    H = dev(ndf.footprint_histograms(*ndf.bin_index(synth.make_map(w), B), L, B), torch.int32)
    init = synth.init_factors(N, L, B, R, 2001)
    ws = g.CPWorkspace(N, L, B, R, "fp32")
    ws.prepare(hist=H)
    fa = g.init_factors_to_device(init)
    fits_a, _ = ws.sweeps(fa, 6)
    fb = g.init_factors_to_device(init)
    fits_b1, _ = ws.sweeps(fb, 3)
    saved = {k: v.clone() for k, v in fb.items()}  # checkpoint
    fc = {k: v.clone() for k, v in saved.items()}
    fits_b2, _ = ws.sweeps(fc, 3)
    assert fits_a[:3] == fits_b1
    assert fits_a[3:] == fits_b2
    for k in fa:
        assert torch.equal(fa[k], fc[k])


GOLDEN_512 = os.path.join(os.path.dirname(__file__), "golden", "brushed512_als_fits.txt")


@pytest.mark.parametrize("prec,tol", [("bf16", 1e-4), ("tf32", 2e-4), ("fp32", 1e-5)])
def test_als_brushed512_full_size_vs_fp64_oracle(prec, tol):
    # the 512^2 precision workload: 20 sweeps from the shared seeded init, the
    # NDF tensor built on the GPU straight from the normal map; the FP64
    # oracle's fits come from tests/golden/make_brushed512_fits.py
    import paper_2109_14807_gb300 as g
    w = synth.WORKLOADS["brushed512"]
    N, L, B, R, sweeps = w["N"], w["levels"], w["bins"], w["rank"], w["sweeps"]
    ref = np.loadtxt(GOLDEN_512, comments="#")[:, 1]
    m = dev(synth.make_map(w))
    init = synth.init_factors(N, L, B, R, 2000 + w["seed"])
    _, fits, _ = g.cp_decompose(R, init, normal_xy=m, levels=L, bins=B, sweeps=sweeps, precision=prec)
    rel = np.abs(np.array(fits) - ref) / np.abs(ref)
    assert np.max(rel) <= tol, (prec, np.max(rel), fits[-1], ref[-1])
    torch.cuda.empty_cache()


def test_solve_reciprocal_is_within_one_ulp():
    # the Cholesky pivot reciprocal (Newton-Raphson from the FP32 reciprocal)
    # against the correctly rounded 1/d, over a log-uniform range and the edges
    # of its fast path
    import paper_2109_14807_gb300 as g
    u = synth.uniform(17, 0, 200_000)
    d = 10.0 ** (60 * u - 30)
    d = np.concatenate([d, [1.0, 2.0, 0.5, 3.0, 1e-30, 1.0000001e-30, 9.999e29, 1e30, 1e-300, 1e300,
                            np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0)]])
    got = g.selftest_recip(dev(d, torch.float64)).cpu().numpy()
    ref = 1.0 / d
    assert np.all(np.abs(got - ref) <= np.spacing(ref)), np.max(np.abs(got - ref) / np.spacing(ref))
    assert g.selftest_recip(dev(d[:0], torch.float64)).numel() == 0


@pytest.mark.parametrize("prec", ["bf16", "fp32", "tf32"])
def test_workspace_sized_by_occupied_bins(prec):
    # a workspace sized for the bins that occur gives bit-identical sweeps to
    # one sized for all B^2 bins; one sized for fewer bins than occur is
    # refused by the prepare
    import paper_2109_14807_gb300 as g
    from paper_2109_14807_gb300._lib import GspError
    N, L, B, R = 64, 7, 32, 16
    if not _supported(prec, N, L, B, R):
        pytest.skip(f"{prec} path unavailable")
    m = synth.flake_map(N, 1000, 0.6, 3)  # 389 of the 1024 bins occur
    s, t = ndf.bin_index(m, B)
    n_occ = len(np.unique(s * B + t))
    assert 256 < n_occ < 512
    md = dev(m)
    assert g.count_bins(L, B, normal_xy=md) == n_occ
    H = g.build_footprint_ndfs(md, L, B)
    assert g.count_bins(L, B, hist=H) == n_occ
    small = g.CPWorkspace.for_map(L, B, R, prec, normal_xy=md)
    full = g.CPWorkspace(N, L, B, R, prec)
    assert small.buf.numel() < full.buf.numel()
    init = synth.init_factors(N, L, B, R, 5)
    fits = []
    for ws in (small, full):
        ws.prepare(normal_xy=md)
        f = g.init_factors_to_device(init)
        fits.append(ws.sweeps(f, 3)[0])
    assert fits[0] == fits[1]
    tight = g.CPWorkspace(N, L, B, R, prec, occupied_bins=200)  # 256 columns instead of 384
    with pytest.raises(GspError) as e:
        tight.prepare(normal_xy=md)
    assert e.value.code == -3


def test_bench_shape_workspace_is_a_few_gb():
    # the 1024^2 flake map with 11 levels and 32^2 bins (67 occur) at rank 64:
    # BF16 operand 1.85 GB, the whole workspace under 4 GB instead of 23 GB
    from paper_2109_14807_gb300 import _lib
    lib_ = _lib.load()
    w = synth.WORKLOADS["flakes1024"]
    m = dev(synth.make_map(w))
    import paper_2109_14807_gb300 as g
    n = g.count_bins(w["levels"], w["bins"], normal_xy=m)
    s, t = ndf.bin_index(synth.make_map(w), w["bins"])
    assert n == len(np.unique(s * w["bins"] + t))
    nb = lib_.gsp_cp_workspace_bytes_for_bins(w["N"], w["levels"], w["bins"], w["rank"],
                                              _lib.PREC["bf16"], n)
    assert 0 < nb < 4 << 30


@pytest.mark.parametrize("prec", ["fp32", "structured"])
def test_singular_gram_system_takes_the_pseudo_inverse(prec):
    # every texel has the same normal, so T = B^2/4 e_b (x) e_b on every footprint:
    # an exactly rank-1 tensor.  After the first sweep the x, y, s and t factors
    # have rank 1, so the Hadamard products of the Gram matrices have rank at
    # most L < R: the Cholesky must fail and the update comes from the Jacobi
    # pseudo-inverse (a numeric fallback).  The factors still fit the tensor:
    # the residual of their reconstruction, computed explicitly on the dense
    # tensor, is at FP32 level.  The fit the sweeps report comes from the Gram
    # formula 1 - sqrt(|T|^2 + |T^|^2 - 2 <T, T^>) / |T|, which cancels near a
    # fit of 1: FP32-level MTTKRP rounding (~1e-7) leaves it within ~1e-3 of the
    # FP64 oracle's CP-ALS (numpy pinv), which reaches 1.
    import paper_2109_14807_gb300 as g
    N, L, B, R, sweeps = 16, 5, 8, 16, 4
    m = np.zeros((N, N, 2), dtype=np.float32)
    m[..., 0], m[..., 1] = 0.3, -0.2
    s, t = ndf.bin_index(m, B)
    assert len(np.unique(s * B + t)) == 1
    X = ndf.logical(ndf.normalised_tensor(ndf.footprint_histograms(s, t, L, B), B))
    init = synth.init_factors(N, L, B, R, 4100)
    _, _, ofits = _oracle_fits(X, R, init, sweeps)
    f, fits, fb = g.cp_decompose(R, init, normal_xy=dev(m), levels=L, bins=B, sweeps=sweeps,
                                 precision=prec)
    assert fb > 0
    assert np.max(np.abs(np.array(fits) - ofits)) <= 2e-3, (fits, ofits)
    fd = {k: v.double().cpu().numpy() for k, v in f.items()}
    That = cp.reconstruct(fd["lambda"], [fd[k] for k in ("fx", "fy", "fl", "fs", "ft")])
    resid = np.linalg.norm((X - That).ravel()) / np.linalg.norm(X.ravel())
    assert resid <= 1e-5, resid
