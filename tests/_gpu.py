"""Helpers shared by the GPU parity tests (not collected by pytest)."""
import numpy as np
import torch

import synth
from oracle import query as oq

QUERY_TOL = 1e-5  # kappa-relative error of a CP range query vs the FP64 oracle


def lib():
    from paper_2109_14807_gb300 import _lib, build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return _lib.load()


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def random_factors(N, L, B, R, seed, signed=True):
    """FP32 factors in [-1, 1) (or [0, 1)), lambda in [0.5, 1.5)."""
    out = {}
    for i, (k, n) in enumerate((("fx", N), ("fy", N), ("fl", L), ("fs", B), ("ft", B))):
        u = synth.uniform(seed, 40 + i, n * R).reshape(n, R)
        out[k] = (2 * u - 1 if signed else u).astype(np.float32)
    out["lambda"] = (0.5 + synth.uniform(seed, 49, R)).astype(np.float32)
    return out


def to_device_factors(f):
    return {k: dev(v) for k, v in f.items()}


def oracle_material(f):
    """FP64 oracle material from FP32 factors (numpy or torch), lambda folded."""
    g = {k: (v.double().cpu().numpy() if isinstance(v, torch.Tensor) else np.asarray(v, np.float64))
         for k, v in f.items()}
    return dict(fx=g["fx"], fy=g["fy"], flw=g["fl"] * g["lambda"][None, :], fs=g["fs"], ft=g["ft"])


def query_error(got, mats, q):
    """max over queries of |got - ref| / max(|ref|, kappa)."""
    ref = oq.cp_range_query(mats, q)
    kap = oq.condition_scale(mats, q)
    return float(np.max(oq.kappa_relative_error(got, ref, kap))), ref
