"""GPU parity of the clustered compression layout (row f2, Sec. 4.2 and the
block splitting of Sec. 4.4) against the oracle: the layout bit for bit, every
group's CP-ALS against the FP64 oracle's from the same initial factors, and
range queries (integer, fractional, zero-width, across block borders, across
levels, malformed) on the GPU's own factors."""
import numpy as np
import pytest
import torch

import synth
from oracle import clustered as ocl
from oracle import ndf
from _gpu import dev, lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def _case(N, L, B, kind, seed):
    m = synth.flake_map(N, max(4, N * N // 32), 0.3, seed) if kind == "flakes" else \
        synth.brushed_map(N, 0.05, 0.3, 4, seed)
    s, t = ndf.bin_index(m, B)
    Hl = [ndf.level_histograms(s, t, l, B).astype(np.int32) for l in range(L)]
    return m, Hl, dev(np.stack(Hl), torch.int32)


def _oracle_fac(lay_g, fac_g, lay_o):
    """The GPU's factors as the oracle's per-group dict (FP64)."""
    off = lay_g["offsets"].cpu().numpy()
    X = fac_g["X"].double().cpu().numpy()
    Y = fac_g["Y"].double().cpu().numpy()
    Z = fac_g["Z"].double().cpu().numpy()
    lam = fac_g["lam"].double().cpu().numpy()
    return {j: (lam[j], X[j], Y[j], Z[off[j]:off[j + 1]], [])
            for j in range(lay_o["G"]) if off[j + 1] > off[j]}


@pytest.mark.parametrize("N,L,B,kind", [(16, 5, 32, "flakes"), (32, 6, 64, "brushed"), (64, 7, 32, "flakes")])
def test_layout_matches_oracle(N, L, B, kind):
    import paper_2109_14807_gb300 as g
    _, Hl, H = _case(N, L, B, kind, 7 + N)
    lay = g.cluster_layout(H)
    ref = ocl.layout(Hl, B)
    counts = np.array([len(m) for m in ref["members"]])
    assert lay["G"] == ref["G"]
    assert np.array_equal(lay["offsets"].cpu().numpy(), np.concatenate([[0], np.cumsum(counts)]))
    assert lay["total"] == counts.sum() and lay["max_members"] == counts.max()
    assert np.array_equal(lay["zmap"].cpu().numpy(), ref["zmap"])
    mem = lay["members"].cpu().numpy()
    packed = [(l << 20) | (y << 10) | x for m in ref["members"] for (l, y, x) in m]
    assert np.array_equal(mem, np.array(packed, dtype=np.int64))


@pytest.mark.parametrize("R", [8, 16])
def test_group_als_matches_oracle(R):
    import paper_2109_14807_gb300 as g
    N, L, B, sweeps = 16, 5, 32, 6
    _, Hl, H = _case(N, L, B, "flakes", 3)
    lay = g.cluster_layout(H)
    ref = ocl.layout(Hl, B)
    off = lay["offsets"].cpu().numpy()
    X0, Y0, Z0 = synth.cluster_init(lay["G"], off, R, 11)
    st = g.new_status()
    fac = g.cluster_decompose(H, lay, R, (X0, Y0, Z0), max_sweeps=sweeps, tol=0.0, status=st)
    assert g.status_bits(st) & ~0x4 == 0
    init = {j: (X0[j], Y0[j], Z0[off[j]:off[j + 1]]) for j in range(lay["G"]) if off[j + 1] > off[j]}
    ofac = ocl.decompose(Hl, ref, R, init, sweeps)
    fit = fac["fit"].cpu().numpy()
    nsw = fac["sweeps"].cpu().numpy()
    worst = 0.0
    for j, (lam, X, Y, Z, fits) in ofac.items():
        assert nsw[j] == sweeps
        assert abs(fit[j] - fits[-1]) <= 2e-5 * max(1.0, abs(fits[-1])), (j, fit[j], fits[-1])
        # the reconstructed group tensors agree (relative to the data)
        D = ocl.group_tensor(Hl, ref, j)
        gj = _oracle_fac(lay, fac, ref)[j]
        rec_g = np.einsum("r,sr,tr,zr->stz", gj[0], gj[1], gj[2], gj[3])
        rec_o = np.einsum("r,sr,tr,zr->stz", lam, X, Y, Z)
        worst = max(worst, np.linalg.norm(rec_g - rec_o) / np.linalg.norm(D))
    assert worst <= 1e-4, worst
    empty = [j for j in range(lay["G"]) if off[j + 1] == off[j]]
    assert all(nsw[j] == 0 for j in empty)


def test_group_als_stops_at_tolerance():
    import paper_2109_14807_gb300 as g
    N, L, B, R = 16, 5, 32, 8
    _, Hl, H = _case(N, L, B, "brushed", 5)
    lay = g.cluster_layout(H)
    ref = ocl.layout(Hl, B)
    off = lay["offsets"].cpu().numpy()
    X0, Y0, Z0 = synth.cluster_init(lay["G"], off, R, 2)
    fac = g.cluster_decompose(H, lay, R, (X0, Y0, Z0), max_sweeps=200, tol=1e-4)
    nsw = fac["sweeps"].cpu().numpy()
    init = {j: (X0[j], Y0[j], Z0[off[j]:off[j + 1]]) for j in range(lay["G"]) if off[j + 1] > off[j]}
    ofac = ocl.decompose(Hl, ref, R, init, 200, tol=1e-4)
    same = sum(int(nsw[j] == len(v[4])) for j, v in ofac.items())
    # a group whose |delta fit| sits within rounding of the tolerance may stop
    # one sweep apart; all others stop at the same sweep
    assert same >= len(ofac) - 1
    assert all(abs(int(nsw[j]) - len(v[4])) <= 1 for j, v in ofac.items())


def _queries(N, L, B, n, seed):
    q = synth.queries_fractional(N, L, B, n, seed, frac_level=True)
    u = synth.uniform(seed, 77, 4 * n).reshape(n, 4)
    k = np.arange(n) % 6
    # integer, zero-width, whole-image, block-crossing cases
    q["s0"][k == 1] = np.floor(q["s0"][k == 1]); q["s1"][k == 1] = np.ceil(q["s1"][k == 1])
    q["s1"][k == 2] = q["s0"][k == 2]; q["t1"][k == 2] = q["t0"][k == 2]
    q["s0"][k == 3], q["s1"][k == 3], q["t0"][k == 3], q["t1"][k == 3] = 0.0, float(B), 0.0, float(B)
    c = k == 4
    q["s0"][c] = 16.0 - 4.0 * u[c, 0]; q["s1"][c] = 16.0 + 5.0 * u[c, 1]
    q["t0"][c] = 16.0 * u[c, 2]; q["t1"][c] = q["t0"][c] + 20.0 * u[c, 3]
    q["s0"][k == 5] = float(B); q["s1"][k == 5] = float(B)
    return q


@pytest.mark.parametrize("N,L,B,R,kind", [(16, 5, 32, 8, "flakes"), (32, 6, 64, 16, "brushed"),
                                          (64, 7, 32, 32, "flakes")])
def test_cluster_range_query_matches_oracle(N, L, B, R, kind):
    import paper_2109_14807_gb300 as g
    _, Hl, H = _case(N, L, B, kind, 19 + N)
    lay = g.cluster_layout(H)
    ref = ocl.layout(Hl, B)
    off = lay["offsets"].cpu().numpy()
    X0, Y0, Z0 = synth.cluster_init(lay["G"], off, R, 4)
    fac = g.cluster_decompose(H, lay, R, (X0, Y0, Z0), max_sweeps=4, tol=0.0)
    tab = g.cluster_tables(lay, fac)
    q = _queries(N, L, B, 3000, 31)
    st = g.new_status()
    got = g.cluster_range_query(lay, tab, g.queries_to_device(q), status=st).double().cpu().numpy()
    assert g.status_bits(st) == 0
    ofac = _oracle_fac(lay, fac, ref)
    want = ocl.range_query(ref, ofac, q)
    afac = {j: (np.abs(v[0]), np.abs(v[1]), np.abs(v[2]), np.abs(v[3]), []) for j, v in ofac.items()}
    kappa = ocl.range_query(ref, afac, q)
    err = np.abs(got - want) / np.maximum(np.maximum(np.abs(want), kappa), 1e-30)
    assert np.max(err) <= 1e-5, (np.max(err), np.argmax(err))
    # malformed
    bad = q[:2].copy()
    bad["level"][0] = np.nan
    bad["t1"][1] = np.inf
    st = g.new_status()
    o = g.cluster_range_query(lay, tab, g.queries_to_device(bad), status=st).cpu().numpy()
    assert np.all(np.isnan(o)) and g.status_bits(st) & 0x2
