"""GPU parity of the range-query adjoint, the autograd wrapper and Adam (row a7)."""
import numpy as np
import pytest
import torch

import synth
from oracle import query as oq
from _gpu import dev, lib, oracle_material, random_factors

pytestmark = pytest.mark.gpu
NAMES = (("dfx", "fx"), ("dfy", "fy"), ("dflw", "flw"), ("dfs", "fs"), ("dft", "ft"))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


def _gpu_grads(f, q, g_up):
    import paper_2109_14807_gb300 as g
    fd = {k: dev(v) for k, v in f.items()}
    mat = g.QueryMaterial.from_factors(fd)
    g.build_query_tables(mat)
    grads = {k: torch.zeros_like(fd[a if a != "flw" else "fl"]) for k, a in NAMES}
    st = g.new_status()
    g.range_query_backward(mat, g.queries_to_device(q), dev(g_up), [grads], status=st)
    torch.cuda.synchronize()
    assert g.status_bits(st) == 0
    return {k: v.double().cpu().numpy() for k, v in grads.items()}


def _oracle_grad_scale(om, q, g_up):
    """Gradient of sum |g_i| q_i(|factors|): the magnitude the adjoint sums."""
    absm = {k: np.abs(v) for k, v in om.items()}
    return oq.cp_range_query_adjoint(absm, q, np.abs(g_up))


@pytest.mark.parametrize("N,L,B,R", [(16, 5, 8, 8), (64, 7, 32, 16), (32, 6, 16, 64)])
def test_adjoint_matches_fp64_oracle(N, L, B, R):
    f = random_factors(N, L, B, R, 60 + R)
    q = synth.queries_fractional(N, L, B, 3000, 61, wmin=0.05, wmax=B, frac_level=True)
    q[5]["s1"] = q[5]["s0"]  # zero-width sides
    q[9]["t0"] = q[9]["t1"]
    g_up = (synth.uniform(62, 1, len(q)) - 0.5).astype(np.float32)
    got = _gpu_grads(f, q, g_up)
    om = oracle_material(f)
    ref = oq.cp_range_query_adjoint(om, q, g_up.astype(np.float64))
    scale = _oracle_grad_scale(om, q, g_up.astype(np.float64))
    for k, a in NAMES:
        err = np.max(np.abs(got[k] - ref[a]) / np.maximum(scale[a], 1e-30))
        assert err <= 1e-4, (k, err)


def test_adjoint_two_materials_and_malformed_queries():
    # queries of two materials (ranks 16 and 64) in one launch, with malformed
    # ones mixed in: each material's gradients are the oracle's adjoint of its
    # own well-formed queries, and the malformed ones only raise the status bit
    import paper_2109_14807_gb300 as g
    shapes = [(32, 6, 16, 16), (64, 7, 32, 64)]
    fs = [random_factors(N, L, B, R, 70 + i) for i, (N, L, B, R) in enumerate(shapes)]
    parts = []
    for i, (N, L, B, R) in enumerate(shapes):
        qi = synth.queries_fractional(N, L, B, 2000 + 37 * i, 71 + i, frac_level=True)
        qi["material"] = i
        parts.append(qi)
    q = np.concatenate(parts)
    q = q[np.argsort(synth.uniform(72, 0, len(q)))]  # interleave the materials
    q["level"][3] = np.nan
    q["material"][40] = 7  # no such material
    q["t1"][41] = np.inf
    q["s0"][999] = -np.inf
    g_up = (synth.uniform(73, 1, len(q)) - 0.5).astype(np.float32)
    mats, grads = [], []
    for f in fs:
        fd = {k: dev(v) for k, v in f.items()}
        mat = g.QueryMaterial.from_factors(fd)
        g.build_query_tables(mat)
        mats.append(mat)
        grads.append({k: torch.zeros_like(fd[a if a != "flw" else "fl"]) for k, a in NAMES})
    st = g.new_status()
    g.range_query_backward(mats, g.queries_to_device(q), dev(g_up), grads, status=st)
    torch.cuda.synchronize()
    assert g.status_bits(st) & 0x2
    # the oracle takes the material list and skips the malformed queries itself
    oms = [oracle_material(f) for f in fs]
    g64 = g_up.astype(np.float64)
    ref = oq.cp_range_query_adjoint(oms, q, g64)
    scale = oq.cp_range_query_adjoint([{k: np.abs(v) for k, v in om.items()} for om in oms], q, np.abs(g64))
    for i in range(len(fs)):
        for k, a in NAMES:
            got = grads[i][k].double().cpu().numpy()
            err = np.max(np.abs(got - ref[i][a]) / np.maximum(scale[i][a], 1e-30))
            assert err <= 1e-4, (i, k, err)


@pytest.mark.parametrize("ranks", [(32, 64), (64, 64, 32)])
def test_packed_adjoint_several_materials_of_one_rank_block(ranks):
    # materials whose ranks share the 32-rank block run the packed-query
    # kernel (several queries per warp, one table copy per lane group):
    # the same oracle parity, with zero-width and malformed queries mixed in
    import paper_2109_14807_gb300 as g
    shapes = [(32 << i, 6 + i, 16 * (1 + i % 2), R) for i, R in enumerate(ranks)]
    fs = [random_factors(N, L, B, R, 80 + i) for i, (N, L, B, R) in enumerate(shapes)]
    parts = []
    for i, (N, L, B, R) in enumerate(shapes):
        qi = synth.queries_fractional(N, L, B, 1500 + 11 * i, 81 + i, wmin=0.05, wmax=B, frac_level=True)
        qi["material"] = i
        parts.append(qi)
    q = np.concatenate(parts)
    q = q[np.argsort(synth.uniform(82, 0, len(q)))]
    q["s1"][10] = q["s0"][10]
    q["t0"][11] = q["t1"][11]
    q["level"][12] = np.nan
    g_up = (synth.uniform(83, 1, len(q)) - 0.5).astype(np.float32)
    g_up[100:140] = 0.0  # zero upstream gradients: skipped queries
    mats, grads = [], []
    for f in fs:
        fd = {k: dev(v) for k, v in f.items()}
        mat = g.QueryMaterial.from_factors(fd)
        g.build_query_tables(mat)
        mats.append(mat)
        grads.append({k: torch.zeros_like(fd[a if a != "flw" else "fl"]) for k, a in NAMES})
    st = g.new_status()
    g.range_query_backward(mats, g.queries_to_device(q), dev(g_up), grads, status=st)
    torch.cuda.synchronize()
    assert g.status_bits(st) & 0x2
    oms = [oracle_material(f) for f in fs]
    g64 = g_up.astype(np.float64)
    ref = oq.cp_range_query_adjoint(oms, q, g64)
    scale = oq.cp_range_query_adjoint([{k: np.abs(v) for k, v in om.items()} for om in oms], q, np.abs(g64))
    for i in range(len(fs)):
        for k, a in NAMES:
            got = grads[i][k].double().cpu().numpy()
            err = np.max(np.abs(got - ref[i][a]) / np.maximum(scale[i][a], 1e-30))
            assert err <= 1e-4, (ranks, i, k, err)


def test_packed_and_rank_lane_adjoints_agree():
    # the same material with 16-byte aligned factor rows (packed-query kernel)
    # and with factor storage 4 bytes off alignment (the kernel that gives each
    # query a whole warp, one rank per lane): both match the oracle and each other
    import paper_2109_14807_gb300 as g
    N, L, B, R = 64, 7, 32, 64
    f = random_factors(N, L, B, R, 90)
    q = synth.queries_fractional(N, L, B, 4000, 91, wmin=0.05, wmax=B, frac_level=True)
    g_up = (synth.uniform(92, 1, len(q)) - 0.5).astype(np.float32)
    qd, gd = g.queries_to_device(q), dev(g_up)
    out = []
    for shift in (0, 1):
        fd = {}
        for k, v in f.items():
            if shift and k in ("fx", "fy"):
                buf = torch.zeros(v.size + 1, dtype=torch.float32, device="cuda")
                buf[1:] = dev(v).reshape(-1)
                fd[k] = buf[1:].view(v.shape)  # rows 4 bytes off a 16-byte boundary
            else:
                fd[k] = dev(v)
        mat = g.QueryMaterial.from_factors(fd)
        g.build_query_tables(mat)
        grads = {k: torch.zeros(fd[a if a != "flw" else "fl"].shape, dtype=torch.float32, device="cuda")
                 for k, a in NAMES}
        g.range_query_backward(mat, qd, gd, [grads])
        torch.cuda.synchronize()
        out.append({k: v.double().cpu().numpy() for k, v in grads.items()})
    om = oracle_material(f)
    ref = oq.cp_range_query_adjoint(om, q, g_up.astype(np.float64))
    scale = _oracle_grad_scale(om, q, g_up.astype(np.float64))
    for k, a in NAMES:
        for o in out:
            assert np.max(np.abs(o[k] - ref[a]) / np.maximum(scale[a], 1e-30)) <= 1e-4, k
        assert np.max(np.abs(out[0][k] - out[1][k]) / np.maximum(scale[a], 1e-30)) <= 2e-4, k


def test_adjoint_vs_fp32_central_differences():
    import paper_2109_14807_gb300 as g
    N, L, B, R = 16, 5, 8, 8
    f = random_factors(N, L, B, R, 5)
    q = synth.queries_fractional(N, L, B, 500, 6, wmin=0.25, wmax=8, frac_level=True)
    qd = g.queries_to_device(q)
    g_up = (synth.uniform(7, 1, len(q)) - 0.5).astype(np.float32)
    got = _gpu_grads(f, q, g_up)
    gd = dev(g_up)

    def loss(ff):
        mat = g.QueryMaterial.from_factors({k: dev(v) for k, v in ff.items()})
        g.build_query_tables(mat)
        return float((g.range_query(mat, qd).double() * gd.double()).sum())

    h = 1e-3
    u = synth.uniform(8, 8, 40)
    for i, (k, a) in enumerate(NAMES):
        src = "fl" if a == "flw" else a
        for j in range(8):
            idx = np.unravel_index(int(u[i * 8 + j] * f[src].size), f[src].shape)
            fp = {kk: vv.copy() for kk, vv in f.items()}
            fm = {kk: vv.copy() for kk, vv in f.items()}
            # perturb flw = fl * lambda through fl, so divide the step by lambda
            step = h / (f["lambda"][idx[1]] if a == "flw" else 1.0)
            fp[src][idx] += step
            fm[src][idx] -= step
            fd = (loss(fp) - loss(fm)) / (2 * h)
            # FP32 rounding of each query (~6e-8 |q|) divided by h bounds the difference
            assert abs(fd - got[k][idx]) <= 1e-2 * max(1.0, abs(fd)), (k, idx, fd, got[k][idx])


def test_autograd_function_matches_backward():
    import paper_2109_14807_gb300 as g
    N, L, B, R = 32, 6, 16, 16
    f = random_factors(N, L, B, R, 11)
    q = synth.queries_fractional(N, L, B, 4000, 12, frac_level=True)
    qd = g.queries_to_device(q)
    params = [dev(f["fx"]), dev(f["fy"]), dev(f["fl"] * f["lambda"][None]), dev(f["fs"]), dev(f["ft"])]
    for p in params:
        p.requires_grad_(True)
    target = torch.randn(len(q), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    out = g.range_query_autograd(qd, *params)
    loss = ((out - target) ** 2).mean()
    loss.backward()
    om = dict(fx=f["fx"].astype(np.float64), fy=f["fy"].astype(np.float64),
              flw=params[2].detach().double().cpu().numpy(), fs=f["fs"].astype(np.float64),
              ft=f["ft"].astype(np.float64))
    qo = oq.cp_range_query(om, q)
    gup = 2.0 * (qo - target.double().cpu().numpy()) / len(q)
    ref = oq.cp_range_query_adjoint(om, q, gup)
    scale = _oracle_grad_scale(om, q, gup)
    for p, (k, a) in zip(params, NAMES):
        err = np.max(np.abs(p.grad.double().cpu().numpy() - ref[a]) / np.maximum(scale[a], 1e-30))
        assert err <= 1e-4, k


def test_adam_step_matches_formula():
    import paper_2109_14807_gb300 as g
    n = 1000
    p0 = synth.uniform(1, 1, n).astype(np.float32)
    gr = (synth.uniform(1, 2, n) - 0.5).astype(np.float32)
    p, gd = dev(p0), dev(gr)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    pm, mm, vm = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in (1, 2, 3):
        g.adam_step(p, gd, m, v, step, 1e-2)
        mm = 0.9 * mm + 0.1 * gr
        vm = 0.999 * vm + 0.001 * gr.astype(np.float64) ** 2
        pm = pm - 1e-2 * (mm / (1 - 0.9 ** step)) / (np.sqrt(vm / (1 - 0.999 ** step)) + 1e-8)
    assert np.allclose(p.cpu().numpy(), pm, rtol=0, atol=1e-5)


def test_refinement_lowers_range_error():
    # Gradient refinement of ALS factors on range-query error: the plain ALS
    # result is the starting point, Adam steps must not increase the loss.
    import paper_2109_14807_gb300 as g
    from oracle import cp, ndf
    w = synth.WORKLOADS["flakes32"]
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    m = synth.make_map(w)
    s, t = ndf.bin_index(m, B)
    H = ndf.footprint_histograms(s, t, L, B)
    X = ndf.logical(ndf.normalised_tensor(H, B))
    init = synth.init_factors(N, L, B, R, 2001)
    f, _, _ = g.cp_decompose(R, init, hist=dev(H, torch.int32), sweeps=20)
    q = synth.queries_fractional(N, L, B, 20_000, 31, frac_level=True)
    target = dev(oq.dense_range_query(X, q[:20_000]))
    qd = g.queries_to_device(q)
    params = [f["fx"].clone(), f["fy"].clone(), (f["fl"] * f["lambda"][None]).clone(), f["fs"].clone(),
              f["ft"].clone()]
    moments = [(torch.zeros_like(p), torch.zeros_like(p)) for p in params]
    losses = []
    for step in range(1, 31):
        ps = [p.detach().requires_grad_(True) for p in params]
        out = g.range_query_autograd(qd, *ps)
        loss = ((out - target) ** 2).mean()
        loss.backward()
        losses.append(float(loss))
        for p, pg, (mm, vv) in zip(params, ps, moments):
            g.adam_step(p, pg.grad.contiguous(), mm, vv, step, 1e-3)
    assert losses[-1] < losses[0]
