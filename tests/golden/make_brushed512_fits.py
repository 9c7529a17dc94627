"""Write brushed512_als_fits.txt: the FP64 oracle's CP-ALS fit after each of
20 sweeps on the 512^2 brushed-metal workload (levels 0..9, 32 x 32 bins,
rank 32, init seed 2002), the reference the tensor-core and FP32 ALS variants
are compared with.  Calls only the oracle and the input generators.

    python tests/golden/make_brushed512_fits.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import synth  # noqa: E402
from oracle import cp, ndf  # noqa: E402


def main():
    w = synth.WORKLOADS["brushed512"]
    N, L, B, R, sweeps = w["N"], w["levels"], w["bins"], w["rank"], w["sweeps"]
    s, t = ndf.bin_index(synth.make_map(w), B)
    H = [ndf.level_histograms(s, t, l, B).astype(np.int32) for l in range(L)]
    FT = cp.FootprintTensor(H, B)
    f = synth.init_factors(N, L, B, R, 2000 + w["seed"])
    init = [f[k].astype(np.float32).astype(np.float64) for k in ("fx", "fy", "fl", "fs", "ft")]
    t0 = time.time()
    _, _, fits = cp.cp_als(FT, R, init, sweeps, fit_method="gram")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "brushed512_als_fits.txt")
    with open(out, "w") as fh:
        fh.write("# FP64 oracle CP-ALS fits, brushed 512^2 map (sigma 0.05/0.3, 200 scratches,\n")
        fh.write(f"# seed {w['seed']}), levels 0..{L - 1}, {B}x{B} bins, rank {R}, init seed "
                 f"{2000 + w['seed']}, mode order x y l s t; fit = 1 - ||T - That|| / ||T|| after\n")
        fh.write("# each sweep (Sec. 4.2, Eq. 3; Kolda & Bader CP-ALS).  Written by\n")
        fh.write("# tests/golden/make_brushed512_fits.py, which calls only oracle/ and synth.\n")
        for k, v in enumerate(fits):
            fh.write(f"{k + 1} {v:.15f}\n")
    print("wrote", out, f"in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
