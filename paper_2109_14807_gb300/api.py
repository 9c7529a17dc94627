"""Python binding of the C ABI: the same calls, with torch tensors for device
memory and torch's current CUDA stream.  Nothing here computes; every step of
the path runs in libgsp.so.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from ._lib import (AlsOpts, AlsReport, CpFactors, Material, MaterialGrad, QueryTuning, check,
                   load)

QUERY_WORDS = 8  # a query descriptor is 32 bytes = 8 int32 words


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def new_status(device="cuda"):
    """Device status word (uint32 semantics, stored as int32)."""
    return torch.zeros(1, dtype=torch.int32, device=device)


def status_bits(status: torch.Tensor) -> int:
    return int(status.item()) & 0xFFFFFFFF


def queries_to_device(q: np.ndarray, device="cuda") -> torch.Tensor:
    """numpy array of 32-byte descriptors -> int32 tensor [n][8] on the device."""
    words = np.frombuffer(np.ascontiguousarray(q).tobytes(), dtype=np.int32).reshape(-1, QUERY_WORDS)
    return torch.from_numpy(words.copy()).to(device)


# ------------------------------------------------------------ a1 / a2 --

def bin_normals(normal_xy: torch.Tensor, bins: int, status=None) -> torch.Tensor:
    lib = load()
    N = normal_xy.shape[0]
    out = torch.empty((N, N), dtype=torch.int16, device=normal_xy.device)
    check("gsp_bin_normals", lib.gsp_bin_normals(_ptr(normal_xy, torch.float32, "normal_xy"), N,
                                                 bins, _ptr(out), _ptr(status), _stream()))
    return out


def build_footprint_ndfs(normal_xy: torch.Tensor, levels: int, bins: int, out=None, status=None,
                         workspace=None, implicit=False) -> torch.Tensor:
    """int32 histograms [levels][N][N][B][B] (C order [l][y][x][s][t]); with
    `implicit`, no histogram: the bin map int16 [N][N] (s * B + t) in the
    workspace, of which every footprint histogram is a box count."""
    lib = load()
    N = normal_xy.shape[0]
    if implicit:
        out = None
    elif out is None:
        out = torch.empty((levels, N, N, bins, bins), dtype=torch.int32, device=normal_xy.device)
    need = lib.gsp_build_workspace_bytes(N, levels, bins)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=normal_xy.device)
    check("gsp_build_footprint_ndfs", lib.gsp_build_footprint_ndfs(
        _ptr(normal_xy, torch.float32, "normal_xy"), N, levels, bins, _ptr(out, torch.int32, "out"),
        _ptr(workspace), workspace.numel(), _ptr(status), _stream()))
    if implicit:
        return workspace[:N * N * 2].view(torch.int16).view(N, N)
    return out


# ------------------------------------------------------------ a3 / a4 --

FACTOR_NAMES = ("fx", "fy", "fl", "fs", "ft")


def _factors_struct(f: dict) -> CpFactors:
    return CpFactors(*(_ptr(f[k], torch.float32, k) for k in FACTOR_NAMES),
                     _ptr(f["lambda"], torch.float32, "lambda"))


def count_bins(levels, bins, hist=None, normal_xy=None, status=None) -> int:
    """Bins that occur in the normal map (or the level-0 slice of `hist`): the
    count gsp_cp_workspace_bytes_for_bins sizes a workspace by."""
    lib = load()
    src = hist if hist is not None else normal_xy
    N = hist.shape[1] if hist is not None else normal_xy.shape[0]
    ws = torch.empty(max(lib.gsp_cp_count_bins_workspace_bytes(N, bins), 1), dtype=torch.uint8,
                     device=src.device)
    h = ctypes.c_int32()
    check("gsp_cp_count_bins", lib.gsp_cp_count_bins(
        _ptr(hist, torch.int32, "hist"), _ptr(normal_xy, torch.float32, "normal_xy"), N, levels,
        bins, _ptr(ws), ws.numel(), ctypes.byref(h), _ptr(status), _stream()))
    return int(h.value)


class CPWorkspace:
    """Device workspace of one CP decomposition (operand tensor + scratch).
    With `occupied_bins` (from count_bins) it is sized for maps in which that
    many bins occur, else for all B * B bins."""

    def __init__(self, N, levels, bins, rank, precision="fp32", device="cuda", occupied_bins=None):
        lib = load()
        self.N, self.levels, self.bins, self.rank = N, levels, bins, rank
        self.precision = _lib.PREC[precision] if isinstance(precision, str) else int(precision)
        if occupied_bins is None:
            nbytes = lib.gsp_cp_workspace_bytes(N, levels, bins, rank, self.precision)
        else:
            nbytes = lib.gsp_cp_workspace_bytes_for_bins(N, levels, bins, rank, self.precision,
                                                         int(occupied_bins))
        if nbytes == 0:
            raise ValueError("unsupported CP shape")
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)

    @classmethod
    def for_map(cls, levels, bins, rank, precision="fp32", hist=None, normal_xy=None,
                status=None):
        """A workspace sized for the bins that occur in this map."""
        src = hist if hist is not None else normal_xy
        N = hist.shape[1] if hist is not None else normal_xy.shape[0]
        n = count_bins(levels, bins, hist=hist, normal_xy=normal_xy, status=status)
        return cls(N, levels, bins, rank, precision, device=src.device, occupied_bins=n)

    def operand_view(self, nbytes):
        """The first `nbytes` bytes of the prepared operand (uint8 view)."""
        off = load().gsp_cp_operand_offset(self.N, self.levels, self.bins, self.rank,
                                           self.precision)
        return self.buf[off: off + nbytes]

    def _opts(self, sweeps=1, tol=0.0, raw_counts=False):
        return AlsOpts(int(sweeps), self.precision, float(tol), int(bool(raw_counts)), 0)

    def prepare(self, hist=None, normal_xy=None, raw_counts=False, status=None):
        lib = load()
        opts = self._opts(raw_counts=raw_counts)
        check("gsp_cp_prepare", lib.gsp_cp_prepare(
            _ptr(hist, torch.int32, "hist"), _ptr(normal_xy, torch.float32, "normal_xy"),
            self.N, self.levels, self.bins, self.rank, ctypes.byref(opts), _ptr(self.buf),
            self.buf.numel(), _ptr(status), _stream()))

    def operand_cols(self):
        """(bins occurring in the map, operand columns per footprint) of the
        prepared operand (dense-path precisions)."""
        lib = load()
        h = (ctypes.c_int32 * 2)()
        check("gsp_cp_operand_cols", lib.gsp_cp_operand_cols(
            self.N, self.levels, self.bins, self.rank, self.precision, _ptr(self.buf),
            self.buf.numel(), h, _stream()))
        return int(h[0]), int(h[1])

    def sweeps(self, factors: dict, sweeps: int, tol=0.0, report=True):
        """Run ALS sweeps in place on `factors`; returns the list of fits (or None)."""
        lib = load()
        opts = self._opts(sweeps, tol)
        rep = AlsReport() if report else None
        fs = _factors_struct(factors)
        check("gsp_cp_sweeps", lib.gsp_cp_sweeps(
            self.N, self.levels, self.bins, self.rank, ctypes.byref(opts), ctypes.byref(fs),
            ctypes.byref(rep) if rep is not None else None, _ptr(self.buf), self.buf.numel(),
            _stream()))
        if rep is None:
            return None
        return [rep.fit[i] for i in range(rep.sweeps_done)], rep.numeric_fallbacks

    def mttkrp(self, factors: dict):
        """The five MTTKRPs of the prepared operand for fixed factors (FP32)."""
        lib = load()
        dev = self.buf.device
        rows = (self.N, self.N, self.levels, self.bins, self.bins)
        outs = [torch.empty((n, self.rank), dtype=torch.float32, device=dev) for n in rows]
        arr = (ctypes.c_void_p * 5)(*[o.data_ptr() for o in outs])
        f = dict(factors)
        f.setdefault("lambda", torch.ones(self.rank, dtype=torch.float32, device=dev))
        fs = _factors_struct(f)
        check("gsp_cp_mttkrp", lib.gsp_cp_mttkrp(
            self.N, self.levels, self.bins, self.rank, self.precision, ctypes.byref(fs), arr,
            _ptr(self.buf), self.buf.numel(), _stream()))
        return outs


def init_factors_to_device(init: dict, device="cuda") -> dict:
    """numpy init factors (synth.init_factors) -> FP32 device tensors + lambda."""
    out = {k: torch.from_numpy(np.asarray(init[k], dtype=np.float32)).to(device).contiguous()
           for k in FACTOR_NAMES}
    out["lambda"] = torch.ones(out["fx"].shape[1], dtype=torch.float32, device=device)
    return out


def cp_decompose(rank, init: dict, hist=None, normal_xy=None, levels=None, bins=None,
                 sweeps=20, precision="fp32", tol=0.0, raw_counts=False, status=None):
    """CP-ALS of the footprint NDF tensor.  Returns (factors, fits, fallbacks)."""
    src = hist if hist is not None else normal_xy
    if hist is not None:
        levels, N, _, bins, _ = hist.shape
    else:
        N = normal_xy.shape[0]
    ws = CPWorkspace.for_map(levels, bins, rank, precision, hist=hist, normal_xy=normal_xy,
                             status=status)
    ws.prepare(hist=hist, normal_xy=normal_xy, raw_counts=raw_counts, status=status)
    f = init_factors_to_device(init, src.device) if not isinstance(init["fx"], torch.Tensor) else init
    fits, fallbacks = ws.sweeps(f, sweeps, tol)
    return f, fits, fallbacks


# ------------------------------------------------------------ a5 / a6 --

@dataclass
class QueryMaterial:
    """One CP-compressed material: device factor tensors plus its query tables."""
    fx: torch.Tensor
    fy: torch.Tensor
    fl: torch.Tensor
    fs: torch.Tensor
    ft: torch.Tensor
    lam: torch.Tensor
    tables: torch.Tensor = field(default=None)

    @property
    def N(self):
        return self.fx.shape[0]

    @property
    def levels(self):
        return self.fl.shape[0]

    @property
    def bins(self):
        return self.fs.shape[0]

    @property
    def rank(self):
        return self.fx.shape[1]

    def struct(self) -> Material:
        if self.tables is None:
            n = load().gsp_query_table_floats(self.levels, self.bins, self.rank)
            self.tables = torch.empty(n, dtype=torch.float32, device=self.fx.device)
        return Material(self.N, self.levels, self.bins, self.rank,
                        *(_ptr(getattr(self, k), torch.float32, k) for k in
                          ("fx", "fy", "fl", "fs", "ft", "lam")), _ptr(self.tables))

    @staticmethod
    def from_factors(f: dict) -> "QueryMaterial":
        return QueryMaterial(f["fx"], f["fy"], f["fl"], f["fs"], f["ft"], f["lambda"])


def build_query_tables(mat: QueryMaterial) -> None:
    lib = load()
    m = mat.struct()
    check("gsp_build_query_tables", lib.gsp_build_query_tables(ctypes.byref(m), _stream()))


def _mats(materials):
    if isinstance(materials, QueryMaterial):
        materials = [materials]
    arr = (Material * len(materials))(*[m.struct() for m in materials])
    return arr, len(materials)


def range_query(materials, queries: torch.Tensor, out=None, status=None, tuning=None,
                workspace=None) -> torch.Tensor:
    """Batched range queries; `queries` is an int32 [n][8] tensor of descriptors."""
    lib = load()
    arr, nm = _mats(materials)
    n = queries.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=queries.device)
    if workspace is None:
        workspace = torch.empty(16, dtype=torch.uint8, device=queries.device)
    tn = QueryTuning(*tuning) if tuning is not None else None
    check("gsp_range_query", lib.gsp_range_query(
        arr, nm, _ptr(queries, torch.int32, "queries"), n, _ptr(out, torch.float32, "out"),
        _ptr(status), ctypes.byref(tn) if tn is not None else None, _ptr(workspace),
        workspace.numel(), _stream()))
    return out


SAMPLE_WORDS = 4     # a sample descriptor is 16 bytes = 4 int32 words
SAMPLE_UNIFORMS = 8  # uniforms one sample consumes


def samples_to_device(s: np.ndarray, device="cuda") -> torch.Tensor:
    """numpy array of 16-byte sample descriptors (x, y, level, material) ->
    int32 tensor [n][4] on the device."""
    words = np.frombuffer(np.ascontiguousarray(s).tobytes(), dtype=np.int32).reshape(-1, SAMPLE_WORDS)
    return torch.from_numpy(words.copy()).to(device)


def sample_ndf(materials, samples: torch.Tensor, uniforms: torch.Tensor, out=None,
               status=None) -> torch.Tensor:
    """Hierarchical NDF importance sampling (Sec. 5.2): one sample per
    descriptor, consuming uniforms[i] (float32 [n][8] in [0, 1)).  Returns
    float32 [n][4]: s, t (bin units), pmf of the chosen bin, its NDF value."""
    lib = load()
    arr, nm = _mats(materials)
    n = samples.shape[0]
    if uniforms.shape != (n, SAMPLE_UNIFORMS):
        raise ValueError(f"uniforms must be [n][{SAMPLE_UNIFORMS}]")
    if out is None:
        out = torch.empty((n, 4), dtype=torch.float32, device=samples.device)
    check("gsp_sample_ndf", lib.gsp_sample_ndf(
        arr, nm, _ptr(samples, torch.int32, "samples"), n, _ptr(uniforms, torch.float32, "uniforms"),
        _ptr(out, torch.float32, "out"), _ptr(status), _stream()))
    return out


def range_query_interp(materials, queries: torch.Tensor, out=None, status=None, tuning=None,
                       workspace=None) -> torch.Tensor:
    """Range queries at fractional texel positions (descriptors with float x, y,
    int32 [n][8] words): the bilinear blend of the four neighbouring
    footprints' range queries."""
    lib = load()
    arr, nm = _mats(materials)
    n = queries.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=queries.device)
    if workspace is None:
        workspace = torch.empty(16, dtype=torch.uint8, device=queries.device)
    tn = QueryTuning(*tuning) if tuning is not None else None
    check("gsp_range_query_interp", lib.gsp_range_query_interp(
        arr, nm, _ptr(queries, torch.int32, "queries"), n, _ptr(out, torch.float32, "out"),
        _ptr(status), ctypes.byref(tn) if tn is not None else None, _ptr(workspace),
        workspace.numel(), _stream()))
    return out


def env_queries(materials, sgs: torch.Tensor, records: torch.Tensor, eps: float = 0.3,
                out=None) -> torch.Tensor:
    """Range-query descriptors for environment-light prefiltering (Sec. 5.4):
    `sgs` float32 [n_sg][8] (axis x, y, z, amplitude, sharpness, 3 pad),
    `records` int32 [n][8] words of gsp_env_record; returns int32 [n][8]
    query descriptors for range_query."""
    lib = load()
    arr, nm = _mats(materials)
    n = records.shape[0]
    if out is None:
        out = torch.empty((n, QUERY_WORDS), dtype=torch.int32, device=records.device)
    check("gsp_env_queries", lib.gsp_env_queries(
        arr, nm, _ptr(sgs, torch.float32, "sgs"), sgs.shape[0], _ptr(records, torch.int32, "records"),
        n, float(eps), _ptr(out, torch.int32, "out"), _stream()))
    return out


# ------------------------------------------------------------------- f2 --

CLUSTER_BLOCK = 16


def cluster_layout(hist: torch.Tensor) -> dict:
    """The clustered layout (Sec. 4.2) of int32 histograms [L][N][N][B][B]:
    offsets [G+1], members, zmap [L][N][N][nb*nb], total and largest group."""
    lib = load()
    L, N, _, B, _ = hist.shape
    G = lib.gsp_cluster_groups(N, L, B)
    if G == 0:
        raise ValueError("unsupported clustered shape")
    nb = B // CLUSTER_BLOCK
    dev = hist.device
    offsets = torch.empty(G + 1, dtype=torch.int32, device=dev)
    members = torch.empty(L * N * N * nb * nb, dtype=torch.int32, device=dev)
    zmap = torch.empty((L, N, N, nb * nb), dtype=torch.int32, device=dev)
    ws = torch.empty(lib.gsp_cluster_layout_bytes(N, L, B), dtype=torch.uint8, device=dev)
    stats = (ctypes.c_int64 * 2)()
    check("gsp_cluster_layout", lib.gsp_cluster_layout(
        _ptr(hist, torch.int32, "hist"), N, L, B, _ptr(offsets), _ptr(members), _ptr(zmap), stats,
        _ptr(ws), ws.numel(), _stream()))
    total, mmax = int(stats[0]), int(stats[1])
    return dict(N=N, L=L, B=B, nb=nb, G=G, offsets=offsets, members=members[:total], zmap=zmap,
                total=total, max_members=mmax)


def cluster_decompose(hist: torch.Tensor, lay: dict, rank: int, init, max_sweeps=500, tol=1e-4,
                      raw_counts=False, status=None) -> dict:
    """Batched CP-ALS of every group (one CTA per group).  `init` = (X0 [G][16][R],
    Y0 [G][16][R], Z0 [total][R]) (numpy or device tensors); returns the factors,
    lambda [G][R], sweeps [G] and fit [G]."""
    lib = load()
    dev = hist.device

    def _dev(a):
        t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
        return t.to(dev, torch.float32).contiguous().clone()

    X, Y, Z = (_dev(a) for a in init)
    G, L = lay["G"], lay["L"]
    lam = torch.empty((G, rank), dtype=torch.float32, device=dev)
    sweeps = torch.empty(G, dtype=torch.int32, device=dev)
    fit = torch.empty(G, dtype=torch.float64, device=dev)
    ws = torch.empty(max(8 * L, 256), dtype=torch.uint8, device=dev)
    check("gsp_cluster_als", lib.gsp_cluster_als(
        _ptr(hist, torch.int32, "hist"), lay["N"], L, lay["B"], rank, _ptr(lay["offsets"]),
        _ptr(lay["members"]) if lay["total"] else _ptr(lay["offsets"]), lay["max_members"],
        _ptr(X), _ptr(Y), _ptr(Z) if lay["total"] else _ptr(X), _ptr(lam), int(max_sweeps), float(tol),
        int(bool(raw_counts)), _ptr(sweeps), _ptr(fit), _ptr(status), _ptr(ws), ws.numel(), _stream()))
    return dict(X=X, Y=Y, Z=Z, lam=lam, sweeps=sweeps, fit=fit, rank=rank)


def cluster_tables(lay: dict, fac: dict) -> dict:
    """SATs of X and Y per group and lambda-weighted Z rows (Sec. 4.4)."""
    lib = load()
    G, R = lay["G"], fac["rank"]
    dev = fac["X"].device
    xsat = torch.empty((G, CLUSTER_BLOCK + 1, R, 4), dtype=torch.float32, device=dev)
    ysat = torch.empty_like(xsat)
    zw = torch.empty((max(lay["total"], 1), R), dtype=torch.float32, device=dev)
    check("gsp_cluster_tables", lib.gsp_cluster_tables(
        lay["N"], lay["L"], lay["B"], R, _ptr(lay["offsets"]), _ptr(fac["X"]), _ptr(fac["Y"]),
        _ptr(fac["Z"]), _ptr(fac["lam"]), _ptr(xsat), _ptr(ysat), _ptr(zw), _stream()))
    return dict(xsat=xsat, ysat=ysat, zw=zw, rank=R)


def cluster_range_query(lay: dict, tables: dict, queries: torch.Tensor, out=None,
                        status=None) -> torch.Tensor:
    """Range queries (gsp_query descriptors, int32 [n][8]) against the clustered layout."""
    lib = load()
    n = queries.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=queries.device)
    check("gsp_cluster_range_query", lib.gsp_cluster_range_query(
        lay["N"], lay["L"], lay["B"], tables["rank"], _ptr(lay["offsets"]), _ptr(lay["zmap"]),
        _ptr(tables["xsat"]), _ptr(tables["ysat"]), _ptr(tables["zw"]),
        _ptr(queries, torch.int32, "queries"), n, _ptr(out, torch.float32, "out"), _ptr(status),
        _stream()))
    return out


def backward_workspace_bytes(materials) -> int:
    arr, nm = _mats(materials)
    return load().gsp_backward_workspace_bytes(arr, nm)


def range_query_backward(materials, queries, gout, grads, status=None, workspace=None):
    """Accumulate factor gradients: grads[m] = dict(dfx, dfy, dflw, dfs, dft)."""
    lib = load()
    arr, nm = _mats(materials)
    garr = (MaterialGrad * nm)(*[MaterialGrad(*(_ptr(g[k], torch.float32, k) for k in
                                                ("dfx", "dfy", "dflw", "dfs", "dft")))
                                 for g in grads])
    need = lib.gsp_backward_workspace_bytes(arr, nm)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=queries.device)
    check("gsp_range_query_backward", lib.gsp_range_query_backward(
        arr, nm, _ptr(queries, torch.int32, "queries"), queries.shape[0],
        _ptr(gout, torch.float32, "gout"), garr, _ptr(workspace), workspace.numel(), _ptr(status),
        _stream()))


def adam_step(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    lib = load()
    check("gsp_adam_step", lib.gsp_adam_step(_ptr(param, torch.float32), _ptr(grad, torch.float32),
                                             _ptr(m, torch.float32), _ptr(v, torch.float32),
                                             param.numel(), int(step), float(lr), float(beta1),
                                             float(beta2), float(eps), _stream()))


# ----------------------------------------------------------------- a7 --

class RangeQueryFn(torch.autograd.Function):
    """q = range_query(fx, fy, flw, fs, ft; queries) with a hand-written adjoint.

    The CP weights are folded into flw (lambda = 1), the parameterisation the
    query tables use, so gradients come back for all five factor matrices."""

    @staticmethod
    def forward(ctx, queries, fx, fy, flw, fs, ft):
        ones = torch.ones(fx.shape[1], dtype=torch.float32, device=fx.device)
        mat = QueryMaterial(fx.contiguous(), fy.contiguous(), flw.contiguous(), fs.contiguous(),
                            ft.contiguous(), ones)
        build_query_tables(mat)
        out = range_query(mat, queries)
        ctx.mat = mat
        ctx.save_for_backward(queries)
        return out

    @staticmethod
    def backward(ctx, gout):
        (queries,) = ctx.saved_tensors
        mat = ctx.mat
        g = {k: torch.zeros_like(getattr(mat, a)) for k, a in
             (("dfx", "fx"), ("dfy", "fy"), ("dflw", "fl"), ("dfs", "fs"), ("dft", "ft"))}
        range_query_backward(mat, queries, gout.contiguous().float(), [g])
        return None, g["dfx"], g["dfy"], g["dflw"], g["dfs"], g["dft"]


def range_query_autograd(queries, fx, fy, flw, fs, ft):
    return RangeQueryFn.apply(queries, fx, fy, flw, fs, ft)


def selftest_wait_timeout(status: torch.Tensor | None = None) -> torch.Tensor:
    """Run the failure-path self-test of the bounded device waits: one CTA waits
    on an mbarrier nothing arrives at until the wait's clock budget (about 2 s)
    runs out, then raises GSP_DEV_TIMEOUT in `status` (a new zeroed device word
    when None).  Returns the status tensor (read it after synchronising)."""
    lib = load()
    if status is None:
        status = new_status()
    check("gsp_selftest_wait_timeout", lib.gsp_selftest_wait_timeout(_ptr(status), _stream()))
    return status


def selftest_recip(d: torch.Tensor) -> torch.Tensor:
    """The CP-ALS solve's FP64 reciprocal of every element of `d` (device FP64)."""
    lib = load()
    d = d.contiguous()
    out = torch.empty_like(d)
    check("gsp_selftest_recip", lib.gsp_selftest_recip(_ptr(d, torch.float64, "d"), d.numel(),
                                                      _ptr(out, torch.float64), _stream()))
    return out
