"""Gradient refinement at the differentiation workload (row a7): a 256^2 flake
map, levels 0..8, 32 x 32 bins, CP rank 16 from 20 ALS sweeps, then 200 Adam
steps (lr 1e-3) on the mean squared error of 10^6 fractional range queries
against the exact dense range averages of the NDF tensor (the oracle's),
evaluated on 10^5 held-out queries drawn with another seed; the plain ALS
factors are the baseline.  The level slices are counted in a process pool
started with `spawn` (safe whatever the parent has done on the GPU).

The range error is heavy-tailed: on the held-out set the worst 0.1 % of the
queries (mostly footprints below level 1 with ranges about one bin wide over
a texel's own bin, densities up to B^2/4) carry two thirds of the squared
error of the ALS factors, the worst 1 % nine tenths.  200 Adam steps fit those
few thousand training queries (training error 0.40x of the ALS factors') but
not the held-out ones: a sweep of learning rates from 1e-5 to 1e-3 never
lowered the held-out error by more than 0.1 %, and at 1e-3 it rose 1.8x.  So
the test asserts the training reduction (the adjoint and the optimiser work
at this scale) and bounds the held-out error of the refined factors."""
import multiprocessing as mp

import numpy as np
import pytest
import torch

import synth
from oracle import ndf
from oracle import query as oq
from _gpu import dev, lib

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    return lib()


class _LevelRows:
    """The normalised tensor in logical order (x, y, l, s, t), read one
    footprint row T[x, y, l] at a time from the per-level count slices (the
    oracle's dense range query only indexes rows)."""

    def __init__(self, H_levels, bins):
        self.H = H_levels
        self.bins = bins
        N = H_levels[0].shape[0]
        self.shape = (N, N, len(H_levels), bins, bins)

    def __getitem__(self, idx):
        x, y, l = idx
        return self.H[l][y, x].astype(np.float64) * ndf.density_scale(l, self.bins)


def _level_slice(args):
    s, t, l, B = args
    return ndf.level_histograms(s, t, l, B).astype(np.int32)


N_TRAIN, N_HELD_OUT = 1_000_000, 100_000
# training MSE after 200 steps / training MSE of the ALS factors (measured 0.40)
TRAIN_RATIO_BOUND = 0.5
# held-out MSE after 200 steps / held-out MSE of the ALS factors (measured 1.78)
HELD_OUT_RATIO_BOUND = 2.5


def test_refinement_at_differentiation_workload():
    w = synth.WORKLOADS["flakes256"]
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    m = synth.make_map(w)
    s, t = ndf.bin_index(m, B)
    with mp.get_context("spawn").Pool(4) as pool:
        H = pool.map(_level_slice, [(s, t, l, B) for l in range(L)])
    import paper_2109_14807_gb300 as g
    q = synth.queries_fractional(N, L, B, N_TRAIN, 4242, frac_level=True)
    qh = synth.queries_fractional(N, L, B, N_HELD_OUT, 4343, frac_level=True)
    rows = _LevelRows(H, B)
    target = oq.dense_range_query(rows, q)  # exact range averages, FP64
    target_h = oq.dense_range_query(rows, qh)
    assert np.all(np.isfinite(target)) and np.all(np.isfinite(target_h))
    del H, rows

    init = synth.init_factors(N, L, B, R, 2000 + w["seed"])
    f, fits, _ = g.cp_decompose(R, init, normal_xy=dev(m), levels=L, bins=B, sweeps=w["sweeps"],
                                precision="fp32")
    qd, qhd = g.queries_to_device(q), g.queries_to_device(qh)
    tgt, tgt_h = dev(target.astype(np.float32)), dev(target_h.astype(np.float32))
    params = [f["fx"].clone(), f["fy"].clone(), (f["fl"] * f["lambda"][None]).clone(),
              f["fs"].clone(), f["ft"].clone()]

    def held_out_mse(ps):
        with torch.no_grad():
            out = g.range_query_autograd(qhd, *ps)
            return float(((out - tgt_h) ** 2).mean())

    base_h = held_out_mse(params)
    moments = [(torch.zeros_like(p), torch.zeros_like(p)) for p in params]
    losses = []
    for step in range(1, 201):
        ps = [p.detach().requires_grad_(True) for p in params]
        out = g.range_query_autograd(qd, *ps)
        loss = ((out - tgt) ** 2).mean()
        loss.backward()
        losses.append(float(loss.detach()))
        for p, pg, (mm, vv) in zip(params, ps, moments):
            g.adam_step(p, pg.grad.contiguous(), mm, vv, step, 1e-3)
    with torch.no_grad():
        out = g.range_query_autograd(qd, *params)
        final = float(((out - tgt) ** 2).mean())
    final_h = held_out_mse(params)
    print(f"\nALS fit {fits[-1]:.6f}; range MSE on the {N_TRAIN} training queries: ALS "
          f"{losses[0]:.6e} -> {final:.6e} after 200 Adam steps ({final / losses[0]:.3f}x); on the "
          f"{N_HELD_OUT} held-out queries: ALS {base_h:.6e} -> {final_h:.6e} ({final_h / base_h:.3f}x)")
    assert final <= TRAIN_RATIO_BOUND * losses[0], (final, losses[0])
    assert final_h <= HELD_OUT_RATIO_BOUND * base_h, (final_h, base_h)
