"""Write flakes1024_als_fits.txt: the FP64 oracle's CP-ALS fit after each of 5
sweeps on the 1024^2 Voronoi-flake workload (levels 0..10, 32 x 32 bins, rank
64, init seed 2003), with the structured MTTKRP (the footprint window moved
onto the spatial factors; pinned to the dense tensor in
tests/test_oracle_structured.py) and ||T||^2 from the exact chunked sums of
squares of the histogram counts.  Calls only the oracle and the input
generators.

    python tests/golden/make_flakes1024_struct_fits.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import synth  # noqa: E402
from oracle import cp, ndf  # noqa: E402

SWEEPS = 5


def main():
    w = synth.WORKLOADS["flakes1024"]
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    s, t = ndf.bin_index(synth.make_map(w), B)
    t0 = time.time()
    sumsq = [ndf.level_sumsq(s, t, l, B) for l in range(L)]
    SF = cp.StructuredFootprint(s, t, L, B)
    norm2 = float(sum(q * SF.scale[l] ** 2 for l, q in enumerate(sumsq)))
    SF = cp.StructuredFootprint(s, t, L, B, norm2=norm2)
    f = synth.init_factors(N, L, B, R, 2000 + w["seed"])
    init = [f[k].astype("float32").astype("float64") for k in ("fx", "fy", "fl", "fs", "ft")]
    _, _, fits = cp.cp_als(SF, R, init, SWEEPS, fit_method="gram")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flakes1024_als_fits.txt")
    with open(out, "w") as fh:
        fh.write(f"# FP64 oracle CP-ALS fits, Voronoi flakes 1024^2 ({w['cells']} cells, Beckmann "
                 f"alpha {w['alpha']}, seed {w['seed']}),\n")
        fh.write(f"# levels 0..{L - 1}, {B}x{B} bins, rank {R}, init seed {2000 + w['seed']}, mode "
                 "order x y l s t; structured MTTKRP (Sec. 4.1 box\n")
        fh.write("# windows moved onto the spatial factors), fit = 1 - ||T - That|| / ||T|| after "
                 "each sweep (Sec. 4.2, Eq. 3).\n")
        fh.write("# Written by tests/golden/make_flakes1024_struct_fits.py, which calls only "
                 "oracle/ and synth.\n")
        fh.write("# per-level sums of squared counts: " + " ".join(str(q) for q in sumsq) + "\n")
        for k, v in enumerate(fits):
            fh.write(f"{k + 1} {v:.15f}\n")
    print("wrote", out, f"in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
