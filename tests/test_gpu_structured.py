"""GPU parity of the structured CP-ALS path (exact MTTKRP from the bin map,
the footprint window moved onto the spatial factors): the five MTTKRPs element
by element against the FP64 oracle (O7b, itself pinned to the dense tensor),
ALS fits against the oracle's CP-ALS and the brushed 512^2 golden fits, and
the two ways in (normal map, int32 histograms) against each other."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import cp, ndf
from _gpu import dev, lib

pytestmark = pytest.mark.gpu

# error of an MTTKRP entry relative to the same MTTKRP of |factors| (its
# magnitude scale): FP32 products, FP32 sums over at most a row split of
# texels, FP64 beyond
STRUCT_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def _map(N, kind, seed):
    if kind == "flakes":
        return synth.flake_map(N, max(4, N * N // 16), 0.3, seed)
    return synth.brushed_map(N, 0.05, 0.3, 6, seed)


def _factors(N, L, B, R, seed, signed):
    u = [synth.uniform(seed, k, n * R).reshape(n, R) for k, n in enumerate((N, N, L, B, B))]
    return [(2 * a - 1 if signed else a).astype(np.float32) for a in u]


def _check_mttkrp(ws, SF, A32):
    f = {k: dev(a) for k, a in zip(("fx", "fy", "fl", "fs", "ft"), A32)}
    outs = ws.mttkrp(f)
    torch.cuda.synchronize()
    A = [a.astype(np.float64) for a in A32]
    Aabs = [np.abs(a) for a in A]
    worst = 0.0
    for n in range(5):
        ref = SF.mttkrp(A, n)
        scale = SF.mttkrp(Aabs, n)
        got = outs[n].double().cpu().numpy()
        err = np.max(np.abs(got - ref) / np.maximum(scale, 1e-300))
        assert err <= STRUCT_TOL, (n, err)
        worst = max(worst, err)
    return worst


@pytest.mark.parametrize("N,L,B,R,kind,raw", [
    (8, 4, 8, 8, "flakes", False), (32, 6, 16, 8, "flakes", False), (64, 7, 16, 16, "brushed", False),
    (64, 5, 32, 32, "flakes", True), (128, 8, 32, 64, "brushed", False), (256, 9, 32, 16, "flakes", False),
    (128, 6, 128, 64, "flakes", False), (64, 7, 64, 8, "brushed", True)])
def test_structured_mttkrp_matches_oracle(N, L, B, R, kind, raw):
    import paper_2109_14807_gb300 as g
    m = _map(N, kind, 7 + N + L)
    s, t = ndf.bin_index(m, B)
    ws = g.CPWorkspace(N, L, B, R, "structured")
    ws.prepare(normal_xy=dev(m), raw_counts=raw)
    SF = cp.StructuredFootprint(s, t, L, B, raw_counts=raw)
    _check_mttkrp(ws, SF, _factors(N, L, B, R, 90 + R, signed=True))


def test_structured_mttkrp_flakes1024_full_size():
    # the scale workload's shape: 1024^2 Voronoi flakes, levels 0..10, 32 x 32 bins, rank 64
    import paper_2109_14807_gb300 as g
    w = synth.WORKLOADS["flakes1024"]
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    m = synth.make_map(w)
    s, t = ndf.bin_index(m, B)
    ws = g.CPWorkspace(N, L, B, R, "structured")
    assert ws.buf.numel() < 256 << 20  # no tensor: tens of MB instead of 23.6 GB
    ws.prepare(normal_xy=dev(m))
    SF = cp.StructuredFootprint(s, t, L, B)
    _check_mttkrp(ws, SF, _factors(N, L, B, R, 404, signed=True))


def test_structured_matches_dense_fp32_mttkrp():
    # the two GPU paths over the same tensor: dense FP32 contraction of the
    # materialised histograms and the structured passes
    import paper_2109_14807_gb300 as g
    N, L, B, R = 64, 7, 16, 16
    m = _map(N, "flakes", 3)
    A32 = _factors(N, L, B, R, 5, signed=False)
    f = {k: dev(a) for k, a in zip(("fx", "fy", "fl", "fs", "ft"), A32)}
    outs = []
    for prec in ("fp32", "structured"):
        ws = g.CPWorkspace(N, L, B, R, prec)
        ws.prepare(normal_xy=dev(m))
        outs.append([o.double().cpu().numpy() for o in ws.mttkrp(f)])
    for a, b in zip(*outs):
        assert np.max(np.abs(a - b) / np.max(np.abs(b))) <= 2e-5


def test_structured_from_histograms_equals_from_normals():
    import paper_2109_14807_gb300 as g
    N, L, B, R = 64, 7, 16, 16
    m = _map(N, "brushed", 12)
    H = g.build_footprint_ndfs(dev(m), L, B)
    init = synth.init_factors(N, L, B, R, 77)
    f1, fits1, _ = g.cp_decompose(R, init, normal_xy=dev(m), levels=L, bins=B, sweeps=5,
                                  precision="structured")
    f2, fits2, _ = g.cp_decompose(R, init, hist=H, sweeps=5, precision="structured")
    assert fits1 == fits2
    for k in ("fx", "fy", "fl", "fs", "ft", "lambda"):
        assert torch.equal(f1[k], f2[k])
    # a level-0 slice that is not one count per texel is reported
    st = g.new_status()
    bad = H.clone()
    bad[0, 3, 5].zero_()
    g.cp_decompose(R, init, hist=bad, sweeps=1, precision="structured", status=st)
    assert g.status_bits(st) & 0x2


def test_structured_als_matches_oracle():
    import paper_2109_14807_gb300 as g
    N, L, B, R, sweeps = 64, 7, 16, 16, 8
    m = _map(N, "brushed", 21)
    s, t = ndf.bin_index(m, B)
    init = synth.init_factors(N, L, B, R, 2021)
    f, fits, fb = g.cp_decompose(R, init, normal_xy=dev(m), levels=L, bins=B, sweeps=sweeps,
                                 precision="structured")
    assert fb == 0
    SF = cp.StructuredFootprint(s, t, L, B)
    A0 = [init[k].astype(np.float32).astype(np.float64) for k in ("fx", "fy", "fl", "fs", "ft")]
    _, A, ofits = cp.cp_als(SF, R, A0, sweeps, fit_method="gram")
    rel = np.abs(np.array(fits) - np.array(ofits)) / np.abs(np.array(ofits))
    assert np.max(rel) <= 1e-6, rel
    # the same factors, up to FP32 rounding carried through the sweeps
    for k, a in zip(("fx", "fy", "fl", "fs", "ft"), A):
        assert np.max(np.abs(f[k].double().cpu().numpy() - a)) <= 1e-4


def test_structured_als_is_bit_reproducible():
    import paper_2109_14807_gb300 as g
    N, L, B, R = 128, 8, 32, 32
    m = dev(_map(N, "flakes", 5))
    init = synth.init_factors(N, L, B, R, 5)
    runs = [g.cp_decompose(R, init, normal_xy=m, levels=L, bins=B, sweeps=3, precision="structured")
            for _ in range(2)]
    assert runs[0][1] == runs[1][1]
    for k in ("fx", "fy", "fl", "fs", "ft", "lambda"):
        assert torch.equal(runs[0][0][k], runs[1][0][k])


GOLDEN_512 = os.path.join(os.path.dirname(__file__), "golden", "brushed512_als_fits.txt")


def test_structured_als_brushed512_vs_fp64_oracle():
    # the 512^2 precision workload, 20 sweeps from the shared seeded init; the
    # FP64 oracle's fits come from tests/golden/make_brushed512_fits.py
    import paper_2109_14807_gb300 as g
    w = synth.WORKLOADS["brushed512"]
    N, L, B, R, sweeps = w["N"], w["levels"], w["bins"], w["rank"], w["sweeps"]
    ref = np.loadtxt(GOLDEN_512, comments="#")[:, 1]
    init = synth.init_factors(N, L, B, R, 2000 + w["seed"])
    _, fits, _ = g.cp_decompose(R, init, normal_xy=dev(synth.make_map(w)), levels=L, bins=B,
                                sweeps=sweeps, precision="structured")
    rel = np.abs(np.array(fits) - ref) / np.abs(ref)
    print(f"\nstructured brushed512: max rel fit error {np.max(rel):.2e}")
    # exact MTTKRPs; what remains is the FP32 storage of the factors (and FP32
    # operands of the solve's products), carried through 20 sweeps: measured
    # 0.5e-6 .. 1.6e-6 across changes of the solve's rounding order, against
    # 3.8e-6 for the dense FP32 contraction
    assert np.max(rel) <= 5e-6, (np.max(rel), fits[-1], ref[-1])


def test_structured_sweeps_in_a_cuda_graph_match_eager():
    # captured, the sweep runs on the capturing stream alone; replayed it gives
    # the eager (side-stream) result bit for bit
    import paper_2109_14807_gb300 as g
    N, L, B, R = 128, 8, 32, 32
    m = dev(_map(N, "brushed", 8))
    init = synth.init_factors(N, L, B, R, 8)
    ws = g.CPWorkspace(N, L, B, R, "structured")
    ws.prepare(normal_xy=m)
    eager = g.init_factors_to_device(init)
    ws.sweeps(eager, 3, report=False)
    cap = g.init_factors_to_device(init)
    start = {k: v.clone() for k, v in cap.items()}
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            ws.sweeps(cap, 3, report=False)
    torch.cuda.current_stream().wait_stream(s)
    for k in cap:
        cap[k].copy_(start[k])
    graph.replay()
    torch.cuda.synchronize()
    for k in ("fx", "fy", "fl", "fs", "ft", "lambda"):
        assert torch.equal(eager[k], cap[k]), k


# ---------------------------------------------------- Gaussian footprints --

@pytest.mark.parametrize("N,L,B,R,kind,raw", [
    (8, 4, 8, 8, "flakes", False), (32, 6, 16, 8, "flakes", False), (64, 7, 16, 16, "brushed", True),
    (128, 8, 32, 32, "brushed", False), (256, 9, 32, 64, "flakes", False)])
def test_gaussian_mttkrp_matches_oracle(N, L, B, R, kind, raw):
    import paper_2109_14807_gb300 as g
    m = _map(N, kind, 3 + N + L)
    s, t = ndf.bin_index(m, B)
    ws = g.CPWorkspace(N, L, B, R, "structured_gaussian")
    ws.prepare(normal_xy=dev(m), raw_counts=raw)
    SF = cp.StructuredFootprint(s, t, L, B, raw_counts=raw, footprint="gaussian")
    _check_mttkrp(ws, SF, _factors(N, L, B, R, 60 + R, signed=True))


@pytest.mark.parametrize("N,L,B,R,kind", [(64, 7, 16, 16, "brushed"), (128, 8, 32, 16, "flakes")])
def test_gaussian_als_matches_oracle(N, L, B, R, kind):
    # the fits also check ||T||^2 from the same-bin autocorrelation
    import paper_2109_14807_gb300 as g
    sweeps = 6
    m = _map(N, kind, 44)
    s, t = ndf.bin_index(m, B)
    init = synth.init_factors(N, L, B, R, 4044)
    f, fits, fb = g.cp_decompose(R, init, normal_xy=dev(m), levels=L, bins=B, sweeps=sweeps,
                                 precision="structured_gaussian")
    assert fb == 0
    SF = cp.StructuredFootprint(s, t, L, B, footprint="gaussian")
    A0 = [init[k].astype(np.float32).astype(np.float64) for k in ("fx", "fy", "fl", "fs", "ft")]
    _, A, ofits = cp.cp_als(SF, R, A0, sweeps, fit_method="gram")
    rel = np.abs(np.array(fits) - np.array(ofits)) / np.abs(np.array(ofits))
    assert np.max(rel) <= 1e-6, rel
    for k, a in zip(("fx", "fy", "fl", "fs", "ft"), A):
        assert np.max(np.abs(f[k].double().cpu().numpy() - a)) <= 1e-4


def test_gaussian_rejects_histograms():
    import paper_2109_14807_gb300 as g
    from paper_2109_14807_gb300._lib import GspError
    N, L, B, R = 32, 6, 16, 8
    H = g.build_footprint_ndfs(dev(_map(N, "flakes", 1)), L, B)
    with pytest.raises(GspError):
        g.cp_decompose(R, synth.init_factors(N, L, B, R, 1), hist=H, sweeps=1,
                       precision="structured_gaussian")


GOLDEN_1024 = os.path.join(os.path.dirname(__file__), "golden", "flakes1024_als_fits.txt")


def test_structured_als_flakes1024_vs_fp64_oracle():
    # the 1024^2 scale workload, 5 sweeps from the shared seeded init; the FP64
    # oracle's fits (structured MTTKRP, exact ||T||^2) come from
    # tests/golden/make_flakes1024_struct_fits.py
    import paper_2109_14807_gb300 as g
    w = synth.WORKLOADS["flakes1024"]
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    ref = np.loadtxt(GOLDEN_1024, comments="#")[:, 1]
    init = synth.init_factors(N, L, B, R, 2000 + w["seed"])
    _, fits, _ = g.cp_decompose(R, init, normal_xy=dev(synth.make_map(w)), levels=L, bins=B,
                                sweeps=len(ref), precision="structured")
    rel = np.abs(np.array(fits) - ref) / np.abs(ref)
    print(f"\nstructured flakes1024: max rel fit error {np.max(rel):.2e}")
    # the first sweep agrees to 1e-7 (exact MTTKRPs, exact ||T||^2); after it the
    # rank-64 ALS amplifies FP32-level rounding: the FP64 oracle itself moves by
    # up to 9.1e-6 over these 5 sweeps when every MTTKRP is perturbed by 1e-7
    # relative noise (and by 1e-9 when only the factors are stored in FP32), so
    # the bound is 3e-5, a third of the 1e-4 asked of the BF16 path
    assert rel[0] <= 1e-6, rel
    assert np.max(rel) <= 3e-5, (np.max(rel), fits, ref)
