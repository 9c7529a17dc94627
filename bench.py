#!/usr/bin/env python3
"""Benchmark of the whole hot path on the 1024^2 metallic-flake workload.

One step = one pass of every row of the path over one batch of synthetic input:
  a1-a3  bin the 1024^2 normal map and build the 11-level footprint NDF tensor
         (1024 x 1024 x 11 x 32 x 32, ~11.8G entries) straight into the MTTKRP
         operand (int32 counts never stored whole);
  a4     one CP-ALS sweep at rank 64 (two MTTKRP passes + FP64 solves);
  a5     query tables (level factor with weights folded in, 1D SATs);
  a6     10^7 range queries with fractional bin rectangles (widths log-uniform
         in [0.5, 16] bins);
  a7     adjoint of the 10^7 queries plus one Adam step on the five factors.
value = range queries per second of whole steps (10^7 / step time).

`--impl reference` times the CPU oracle (FP64 numpy) on a bounded sample of the
same step and extrapolates to the full step.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "NDF range queries/s at 1e-5 rel err; CP-ALS sweep s; % HBM / tensor roofline"
WORKLOAD = "flakes1024"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "kernel_traffic.txt")
ONCHIP_FILE = os.path.join(ROOT, "profiles", "query_onchip_counters.txt")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def parse_args():
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["gsp", "reference"], default="gsp")
    p.add_argument("--precision", choices=["auto", "bf16", "tf32", "fp32"], default="auto")
    p.add_argument("--workload", choices=["flakes1024", "flakes256", "brushed512"],
                   default="flakes1024",
                   help="flakes1024 is the benchmark; the others are smaller cases of the "
                        "same step for profiling")
    p.add_argument("--query-tuning", default=None,
                   help="lanes,blocks_per_sm,threads,chunk for the query kernel instead of the "
                        "autotuner's choice")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp32-sweep", action="store_true",
                   help="skip timing the FP32 CUDA-core sweep after the timed region")
    p.add_argument("--query-profile", action="store_true",
                   help="instead of the step: the query tables, the range queries and their "
                        "adjoint of the workload alone (rank-64 material from the seeded initial "
                        "factors, no NDF tensor), a few hundred MB on the device: the case the "
                        "query kernels' single-kernel ncu captures run")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--report-precisions", default="fp32,tf32,bf16,bf16_1x,structured,structured_gaussian",
                   help="precisions the precision report covers (comma-separated)")
    p.add_argument("--report-workloads", default="brushed512,flakes1024",
                   help="workloads the precision report covers (comma-separated)")
    p.add_argument("--clustered-workload", choices=["clustered256", "clustered64"],
                   default="clustered256",
                   help="workload of --clustered-report (clustered64: a small case for profiling)")
    p.add_argument("--env-report", action="store_true",
                   help="instead of the step: environment-light prefiltering (Sec. 5.4): 10^7 "
                        "shading records against 64 SG lobes turned into range queries and "
                        "answered on the 1024^2 material")
    p.add_argument("--clustered-report", action="store_true",
                   help="instead of the step: the clustered compression layout of Sec. 4.2 on a "
                        "256^2 flake map with 64^2 bins (layout, per-group CP-ALS, compression, "
                        "block-splitting range queries)")
    p.add_argument("--precision-report", action="store_true",
                   help="instead of the step: CP-ALS fit error vs the FP64 oracle and sweep time "
                        "per MTTKRP precision on the 512^2 precision workload, and the sweep time "
                        "per precision on the benchmark workload")
    p.add_argument("--batching-report", action="store_true",
                   help="instead of the step: 8 materials (maps 128-1024, ranks 16-64, bins "
                        "16-64) queried together by 5e7 camera-sweep queries through the "
                        "autotuned, graph-captured query kernel")
    p.add_argument("--sampling-report", action="store_true",
                   help="instead of the step: hierarchical NDF importance sampling (Sec. 5.2) of "
                        "1e7 footprints of the 1024^2, rank-64, 32^2-bin material")
    return p.parse_args()


def workload(name=None):
    global WORKLOAD
    if name:
        WORKLOAD = name
    w = dict(synth.WORKLOADS[WORKLOAD])
    w.setdefault("queries", 1_000_000)
    return w


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- roofline --
def load_peaks():
    try:
        with open(PEAKS_FILE) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


def _code_only(text):
    """C++ source without its comments and blank space, so that an edit of a
    comment does not void a measurement of unchanged code."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def _src_hash(names):
    """sha256 prefix of the code (comments stripped) of the sources `names`
    (csrc file names)."""
    h = hashlib.sha256()
    try:
        for name in names:
            with open(os.path.join(ROOT, "paper_2109_14807_gb300", "csrc", name)) as fh:
                h.update(_code_only(fh.read()).encode())
    except OSError:
        return None
    return h.hexdigest()[:12]


# The source files that fix a kernel's DRAM traffic: its own, plus, for the
# operand kernels, the operand layout (columns kept, tile shapes).
_OPERAND = ("als.cu", "mttkrp.cuh")
KERNEL_SOURCE = {"box_hist": ("binning.cu",) + _OPERAND, "cast": ("als.cu", "mttkrp.cuh"),
                 "mttkrp_xy": ("mttkrp_tc.cu",) + _OPERAND, "mttkrp_lst": ("mttkrp_tc.cu",) + _OPERAND,
                 "range_query": ("query.cu",), "range_query_backward": ("query.cu",)}


def ncu_traffic(kernel, precision):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None
    when absent or when the kernel's sources changed since the capture."""
    src = KERNEL_SOURCE.get(kernel)
    if src is None:
        return None
    if precision == "fp32" and kernel.startswith("mttkrp"):
        src = ("mttkrp_simt.cu",) + _OPERAND
    try:
        lines = open(TRAFFIC_FILE).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        if ln.startswith("#") or not ln.strip():
            continue
        parts = ln.split()
        if len(parts) >= 5 and parts[0] == kernel and parts[1] == WORKLOAD and parts[2] == precision:
            return float(parts[3]) if parts[4] == _src_hash(src) else None
    return None


def ncu_onchip(kernel, lanes):
    """L1 data-pipe wavefronts per launch of a query kernel (ncu counter
    l1tex__data_pipe_lsu_wavefronts.sum, single-kernel capture of
    `bench.py --query-profile`) for this workload and lanes per query, or None
    when absent or when query.cu's code changed since the capture."""
    try:
        lines = open(ONCHIP_FILE).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        if ln.startswith("#") or not ln.strip():
            continue
        parts = ln.split()
        if (len(parts) >= 5 and parts[0] == kernel and parts[1] == WORKLOAD
                and parts[2] == str(lanes)):
            return float(parts[3]) if parts[4] == _src_hash(("query.cu",)) else None
    return None


def l1_peak_gbs(n_sm, sm_mhz):
    """L1 data-pipe peak: one 128-byte wavefront per clock per SM."""
    return n_sm * 128.0 * sm_mhz * 1e6 / 1e9


# ------------------------------------------------------------ replicas --
def max_over_ranks(ms: float, world: int, device=None) -> float:
    """Slowest rank's time (replicas run independently; no data-path
    collective, only this reduction of the timing)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, ms_per_step: float) -> float:
    """Units all ranks processed per second (weak scaling: fixed work per rank)."""
    return units_per_rank * world / (ms_per_step / 1e3)


# ------------------------------------------------------------------ oracle --
def oracle_sample_step(w, m, q, f_init):
    """Time the FP64 oracle on a bounded sample of one step and extrapolate to
    the full step.  Returns (estimated seconds per full step, description)."""
    from oracle import cp as ocp
    from oracle import ndf, query as oq
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    n_q = len(q)
    crop = 128
    sub = m[:crop, :crop]
    s, t = ndf.bin_index(sub, B)
    t0 = time.perf_counter()
    Hs = [ndf.level_histograms(s, t, l, B) for l in (0, 3, 6)]
    t_hist = (time.perf_counter() - t0) / 3 * (N / crop) ** 2 * L
    FT = ocp.FootprintTensor([Hs[1]], B)
    A = [f_init["fx"][:crop], f_init["fy"][:crop], f_init["fl"][:1], f_init["fs"], f_init["ft"]]
    t0 = time.perf_counter()
    for n in range(5):
        FT.mttkrp(A, n)
    t_sweep = (time.perf_counter() - t0) * (N / crop) ** 2 * L
    mat = dict(fx=f_init["fx"], fy=f_init["fy"], flw=f_init["fl"], fs=f_init["fs"], ft=f_init["ft"])
    nq_s = 100_000
    t0 = time.perf_counter()
    qo = oq.cp_range_query(mat, q[:nq_s])
    t_query = (time.perf_counter() - t0) * n_q / nq_s
    na = 400
    t0 = time.perf_counter()
    oq.cp_range_query_adjoint(mat, q[:na], qo[:na])
    t_adj = (time.perf_counter() - t0) * n_q / na
    total = t_hist + t_sweep + t_query + t_adj
    desc = (f"FP64 numpy oracle on bounded samples of one step, extrapolated by work: histograms of "
            f"levels 0,3,6 of a {crop}^2 crop (x{(N // crop) ** 2 * L / 3:.0f}), the five dense MTTKRPs "
            f"of one level of the crop (x{(N // crop) ** 2 * L}), {nq_s} range queries "
            f"(x{n_q // nq_s}), adjoint of {na} queries (x{n_q // na}); stage s: hist {t_hist:.1f}, "
            f"sweep {t_sweep:.1f}, query {t_query:.1f}, adjoint {t_adj:.1f}")
    return total, desc


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(args.workload)
    m = synth.make_map(w)
    q = synth.queries_fractional(w["N"], w["levels"], w["bins"], w["queries"], 1000 + w["seed"])
    f_init = synth.init_factors(w["N"], w["levels"], w["bins"], w["rank"], 2000 + w["seed"])
    times = []
    desc = ""
    for i in range(args.warmup + args.steps):
        est, desc = oracle_sample_step(w, m, q, f_init)
        if i >= args.warmup:
            times.append(est)
    sec = statistics.median(times)
    value = w["queries"] / sec
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(w, "f64"),
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": host_cores(),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_block(w, prec):
    kind = (f"Voronoi flakes ({w['cells']} cells, Beckmann alpha {w['alpha']})" if w["map"] == "flakes"
            else f"brushed (slope sd {w['sigma_x']}/{w['sigma_y']}, {w['scratches']} scratches)")
    return {"workload": f"{WORKLOAD}: {w['N']}x{w['N']} {kind}, levels 0..{w['levels'] - 1}, "
                        f"{w['bins']}x{w['bins']} bins, CP rank {w['rank']}, "
                        f"{w['queries']} fractional range queries",
            "N": w["N"], "levels": w["levels"], "bins": w["bins"], "rank": w["rank"],
            "queries_per_step": w["queries"], "als_sweeps_per_step": 1,
            "mttkrp_precision": prec, "l2": "inputs larger than L2 (operand tensor >> 129 MB)",
            "parallelism": "replicas"}


# -------------------------------------------------------------------- GPU --
def run_gsp(args, rank, world):
    import torch
    import paper_2109_14807_gb300 as g
    from paper_2109_14807_gb300 import _lib, build

    build.build()
    lib = _lib.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = workload(args.workload)
    N, L, B, R, nq = w["N"], w["levels"], w["bins"], w["rank"], w["queries"]
    prec = args.precision
    if prec == "auto":
        prec = "bf16" if lib.gsp_cp_workspace_bytes(N, L, B, R, _lib.PREC["bf16"]) else "fp32"

    m_np = synth.make_map(w)
    q_np = synth.queries_fractional(N, L, B, nq, 1000 + w["seed"])
    f_init = synth.init_factors(N, L, B, R, 2000 + w["seed"])

    normals = torch.from_numpy(m_np).to(dev)
    qd = g.queries_to_device(q_np, dev)
    out = torch.empty(nq, dtype=torch.float32, device=dev)
    status = g.new_status(dev)
    ws = g.CPWorkspace.for_map(L, B, R, prec, normal_xy=normals)  # sized for the occurring bins
    fac = g.init_factors_to_device(f_init, dev)
    mat = g.QueryMaterial.from_factors(fac)
    mat.struct()
    qws = torch.empty(16, dtype=torch.uint8, device=dev)
    grads = {k: torch.zeros_like(fac[a]) for k, a in
             (("dfx", "fx"), ("dfy", "fy"), ("dflw", "fl"), ("dfs", "fs"), ("dft", "ft"))}
    bws = torch.empty(g.backward_workspace_bytes(mat), dtype=torch.uint8, device=dev)
    flw_view = lambda: mat.tables[: L * R]  # noqa: E731  (flw lives at the head of the tables)
    params = [(fac["fx"], "dfx"), (fac["fy"], "dfy"), (None, "dflw"), (fac["fs"], "dfs"),
              (fac["ft"], "dft")]
    moments = {k: (torch.zeros_like(grads[k]), torch.zeros_like(grads[k])) for _, k in params}
    step_no = [0]
    # launch shape of the query kernel from the autotuner (untimed; results do
    # not depend on it)
    from paper_2109_14807_gb300 import tune
    g.build_query_tables(mat)
    if args.query_tuning:
        q_tuning = tuple(int(v) for v in args.query_tuning.split(","))
    else:
        q_tuning = tune.autotune_query(mat, qd, sample=2_000_000, repeats=2)

    def step(stage_events=None, bufs=None):
        ev = stage_events
        normals_s, qd_s, out_s = bufs if bufs is not None else (normals, qd, out)
        if ev: ev[0].record()
        ws.prepare(normal_xy=normals_s, status=status)                   # a1-a3
        if ev: ev[1].record()
        ws.sweeps(fac, 1, report=False)                                  # a4
        if ev: ev[2].record()
        g.build_query_tables(mat)                                        # a5
        if ev: ev[3].record()
        g.range_query(mat, qd_s, out=out_s, status=status, workspace=qws, tuning=q_tuning)  # a6
        if ev: ev[4].record()
        for v in grads.values():
            v.zero_()
        g.range_query_backward(mat, qd_s, out_s, [grads], status=status, workspace=bws)  # a7
        step_no[0] += 1
        for p, k in params:
            p = flw_view() if p is None else p
            mm, vv = moments[k]
            g.adam_step(p, grads[k], mm, vv, step_no[0], 1e-4)
        if ev: ev[5].record()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # warm-up
    for _ in range(args.warmup):
        step()
    barrier()

    # timed region: device-resident inputs
    n_stage = 6
    stage_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(n_stage)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index)
    clocks.start()
    lib.gsp_profile_reset()
    lib.gsp_profile_enable(1)
    launches0 = lib.gsp_kernel_launches()
    barrier()
    t_start.record()
    for k in range(args.steps):
        step(stage_ev[k])
    t_end.record()
    barrier()
    launches = lib.gsp_kernel_launches() - launches0
    lib.gsp_profile_enable(0)
    clk = clocks.stop()
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), world, dev)
    ms_step = total_ms / args.steps
    stages = {name: statistics.median(stage_ev[k][i].elapsed_time(stage_ev[k][i + 1])
                                      for k in range(args.steps))
              for i, name in enumerate(["ndf_build_ms", "als_sweep_ms", "tables_ms",
                                        "range_query_ms", "adjoint_adam_ms"])}
    prof = {}
    for pid in range(15):
        n_l = _lib.c_int64()
        ms = _lib.c_double()
        _lib.check("gsp_profile_read", lib.gsp_profile_read(pid, n_l, ms))
        if n_l.value:
            prof[lib.gsp_profile_name(pid).decode()] = (n_l.value, ms.value)
    st_bits = g.status_bits(status)

    # roofline of the dominant kernel
    peaks, peak_src = load_peaks()
    n_occ, cols = ws.operand_cols()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = roofline(prof, w, prec, peaks, peak_src, n_occ, cols, n_sm=n_sm, sm_mhz=clk.get("sm_mhz"),
                    lanes={"range_query": q_tuning[0], "range_query_backward": "auto"})

    # the plain FP32 CUDA-core path's sweep on the same operand shape, for the
    # BF16-vs-FP32 comparison (after the timed region)
    fp32_sweep = None
    if rank == 0 and world == 1 and prec != "fp32" and not args.no_fp32_sweep:
        fp32_sweep = time_sweep(g, w, normals, f_init, "fp32", dev)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, g, dev, m_np, q_np, normals, qd, out, step, barrier, world)

    # CPU-baseline leg (the only part of the GPU arm that runs the oracle):
    # the oracle timed on a bounded sample of the step, and a parity gate that
    # checks a sample of this run's queries against it
    cpu, parity = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        parity = query_parity(g, mat, qd, q_np, out, tuning=q_tuning)
        est, desc = oracle_sample_step(w, m_np, q_np, f_init)
        cpu = {"value": nq / est, "unit": "queries/s", "cores": host_cores(), "kind": "oracle",
               "sample": desc}

    if rank == 0:
        qps = lambda k: (nq / (prof[k][1] / prof[k][0] / 1e3) if k in prof else None)  # noqa: E731
        line = {
            "metric": METRIC, "value": whole_job_rate(nq, world, ms_step), "unit": "queries/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": config_block(w, prec),
            "gpu_launches": int(launches),
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in prof.items()},
            "query_tuning": list(q_tuning),
            "device_status": st_bits,
            "roofline": roof,
            # kept last, so that they are inside the tail of the line a log keeps
            "query_parity": parity,
            "stages_ms": {k: round(v, 4) for k, v in stages.items()},
            "range_query_kernel_qps": qps("range_query"),
            "adjoint_kernel_qps": qps("range_query_backward"),
            "als_sweep_s": stages["als_sweep_ms"] / 1e3,
            "als_sweep_s_fp32": fp32_sweep,
        }
        print(json.dumps(line), flush=True)


def time_sweep(g, w, normals, f_init, prec, dev, sweeps=3):
    """Seconds per CP-ALS sweep of `prec` on the step's map (operand prepared
    once, one untimed sweep, then `sweeps` sweeps in one call, CUDA events)."""
    import torch
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    ws = g.CPWorkspace.for_map(L, B, R, prec, normal_xy=normals)
    ws.prepare(normal_xy=normals)
    f = g.init_factors_to_device(f_init, dev)
    ws.sweeps(f, 1, report=False)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    ws.sweeps(f, sweeps, report=False)
    b.record()
    torch.cuda.synchronize(dev)
    del ws
    torch.cuda.empty_cache()
    return a.elapsed_time(b) / sweeps / 1e3


# Per-query gather and update rows of the query kernels (fractional rectangle,
# integer level): fx, fy, flw and the two summed-area-table rows of each end
# of both angular ranges read; the adjoint adds one R-wide update row for every
# row read (dfx, dfy, dflw, dP and df at both ends of both ranges).
QUERY_ROWS = 11
ALG_BYTES_DESC = {
    "box_hist": "NDF tensor of all levels written once in the operand type (|X| x element bytes, "
                "|X| = N^2 x levels x operand columns)",
    "cast": "occupied int32 counts of a histogram slice read and operand slice written",
    "mttkrp_xy": "operand tensor read once (|X| x element bytes) + Y' written (N^2 x R x 4 B)",
    "mttkrp_lst": "operand tensor read once (|X| x element bytes) + Z' written (levels x columns x R x 4 B)",
    "range_query": "11 table rows x R x 4 B + 36 B per fractional query (rows are L1/L2-resident: "
                   "DRAM sees the 36 B)",
    "range_query_backward": "11 table rows read + 11 R-wide gradient rows updated, x R x 4 B, + 36 B "
                            "per query (rows and gradient tables are L1/L2/shared-resident)",
}


QUERY_KERNELS = ("range_query", "range_query_backward")


def roofline(prof, w, prec, peaks, peak_src, n_occ, cols, n_sm=152, sm_mhz=None, lanes=None):
    """Roofline of the dominant kernel (largest share of the timed step) and
    the other modelled kernels.  The operand holds `cols` columns per
    footprint (the n_occ bins occurring in the map, zero-padded), so
    |X| = N^2 * L * cols.  Operand kernels are bound by HBM: algorithmic bytes
    per launch / average launch time against the measured copy peak.  The
    query kernels read table rows that stay in L1/L2 (DRAM sees the 36-byte
    descriptor and result): their binding unit is the L1 data pipe, so they
    report L1 wavefronts (counted by ncu for the same code and launch shape)
    x 128 B / live launch time against one wavefront per clock per SM at the
    median SM clock of the timed region; the gather bytes of the query
    definition are kept beside it as a ratio to the HBM peak."""
    N, L, B, R, nq = w["N"], w["levels"], w["bins"], w["rank"], w["queries"]
    esize = 2 if prec == "bf16" else 4
    X = N * N * L * cols
    per_launch = {
        "box_hist": X * esize, "cast": N * N * (n_occ * 4 + cols * esize),
        "mttkrp_xy": X * esize + N * N * R * 4, "mttkrp_lst": X * esize + L * cols * R * 4,
        "range_query": nq * (QUERY_ROWS * R * 4 + 36),
        "range_query_backward": nq * (2 * QUERY_ROWS * R * 4 + 36),
    }
    hbm = float(peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    hbm_src = f"{peak_src} (MEASURED_PEAKS hbm_gbs)" if peak_src == "measured" else "fallback"
    clk = float(sm_mhz or peaks.get("sm_max_mhz", 2070.0))
    l1 = l1_peak_gbs(n_sm, clk)
    lanes = lanes or {}

    def entry(k):
        n_l, ms = prof[k]
        avg_s = ms / n_l / 1e3
        achieved = per_launch[k] / avg_s / 1e9
        if k not in QUERY_KERNELS:
            return {"kernel": k, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": ncu_traffic(k, prec),
                    "algorithmic_bytes_per_launch": per_launch[k], "avg_launch_ms": avg_s * 1e3,
                    "peak_source": hbm_src, "bytes_definition": ALG_BYTES_DESC[k]}
        wf = ncu_onchip(k, lanes.get(k))
        l1_gbs = wf * 128.0 / avg_s / 1e9 if wf is not None else None
        return {"kernel": k, "bound": "l1", "achieved": l1_gbs, "peak": l1, "unit": "GB/s",
                "frac": l1_gbs / l1 if l1_gbs is not None else None,
                "traffic": ncu_traffic(k, prec), "l1_wavefronts_per_launch": wf,
                "avg_launch_ms": avg_s * 1e3,
                "peak_source": f"derived: {n_sm} SMs x 128 B/clk x {clk:.0f} MHz",
                "gather_bytes_per_launch": per_launch[k], "gather_gbs": achieved,
                "gather_vs_hbm_peak": achieved / hbm}

    top = max(prof, key=lambda k: prof[k][1]) if prof else None
    if top not in per_launch:
        return None
    out = entry(top)
    out["occupied_bins"], out["operand_columns"] = n_occ, cols
    out["others"] = [{k2: (round(v, 4) if isinstance(v, float) else v) for k2, v in entry(k).items()
                      if k2 in ("kernel", "bound", "achieved", "frac", "traffic", "avg_launch_ms",
                                "gather_vs_hbm_peak")}
                     for k in sorted(per_launch, key=lambda k: -prof.get(k, (1, 0.0))[1])
                     if k in prof and k != top]
    return out


def query_parity(g, mat, qd, q_np, out, n_sample=100_000, tuning=None):
    """Rebuild the tables from the current factors, answer the step's queries
    with the timed launch configuration, and check a sample against the oracle."""
    from oracle import query as oq
    import torch
    g.build_query_tables(mat)
    g.range_query(mat, qd, out=out, tuning=tuning)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    f = {k: getattr(mat, k).double().cpu().numpy() for k in ("fx", "fy", "fl", "fs", "ft", "lam")}
    om = dict(fx=f["fx"], fy=f["fy"], flw=f["fl"] * f["lam"][None], fs=f["fs"], ft=f["ft"])
    idx = np.sort((synth.uniform(77, 1, n_sample) * len(q_np)).astype(np.int64))
    ref = oq.cp_range_query(om, q_np[idx])
    kap = oq.condition_scale(om, q_np[idx])
    err = float(np.max(oq.kappa_relative_error(got[idx], ref, kap)))
    return {"max_kappa_rel_err": err, "sampled": n_sample, "pass_1e-5": err <= 1e-5}


def run_e2e(args, g, dev, m_np, q_np, normals, qd, out, step, barrier, world):
    """The step end to end from pinned host buffers: every step copies its
    normal map and queries to the device and reads its results back.  Two
    device buffer sets alternate, so the copies of step k + 1 (host-to-device
    stream) and the read-back of step k - 1 (device-to-host stream) overlap the
    compute of step k; the timed region spans every copy of every step."""
    import torch
    h_norm = torch.from_numpy(m_np).pin_memory()
    h_q = torch.from_numpy(np.frombuffer(q_np.tobytes(), dtype=np.int32).reshape(-1, 8).copy()).pin_memory()
    h_out = [torch.empty(out.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    bufs = [(normals, qd, out), (torch.empty_like(normals), torch.empty_like(qd), torch.empty_like(out))]
    comp = torch.cuda.current_stream(dev)
    h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    in_ready = [torch.cuda.Event() for _ in range(2)]
    out_ready = [torch.cuda.Event() for _ in range(2)]
    slot_free = [torch.cuda.Event() for _ in range(2)]
    for e in slot_free:
        e.record(comp)

    def e2e_step(k):
        b = k & 1
        d_norm, d_q, d_out = bufs[b]
        with torch.cuda.stream(h2d):
            h2d.wait_event(slot_free[b])  # step k - 2 has read its inputs and results
            d_norm.copy_(h_norm, non_blocking=True)
            d_q.copy_(h_q, non_blocking=True)
            in_ready[b].record(h2d)
        comp.wait_event(in_ready[b])
        step(bufs=bufs[b])
        out_ready[b].record(comp)
        with torch.cuda.stream(d2h):
            d2h.wait_event(out_ready[b])
            h_out[b].copy_(d_out, non_blocking=True)
            slot_free[b].record(d2h)

    def run(n):
        for k in range(n):
            e2e_step(k)
        for e in slot_free:
            comp.wait_event(e)

    run(max(2, args.warmup))
    barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(comp)
    for e in slot_free:  # the first copies start inside the timed region
        e.record(comp)
    run(args.steps)
    b.record(comp)
    barrier()
    ms = a.elapsed_time(b) / args.steps
    nq = q_np.shape[0]
    return {"value": nq * world / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h_norm.numel() * 4 + h_q.numel() * 4),
            "d2h_bytes_per_step": int(h_out[0].numel() * 4),
            "overlap": "two buffer sets; copies on their own streams overlap the previous / next step"}


# --------------------------------------------------------- query profile --
def query_profile(args):
    """The step's query kernels alone (rows a5-a7 without the NDF tensor):
    the workload's material after one structured ALS sweep from the seeded
    init, its query tables, the step's 10^7 fractional range queries and their
    adjoint with the results as upstream gradients.  A few hundred MB on the
    device, so that single-kernel ncu captures of the query kernels run at the
    bench's rank, query count and live-query mix."""
    import torch
    import paper_2109_14807_gb300 as g
    from paper_2109_14807_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    torch.cuda.set_device(0)
    w = workload(args.workload)
    N, L, B, R, nq = w["N"], w["levels"], w["bins"], w["rank"], w["queries"]
    # factors after one ALS sweep from the seeded init, as in the step: the
    # factor rows of angular bins that no texel falls in are then exactly zero,
    # so are the range queries over them and (with the results as upstream
    # gradients) the adjoint skips them as the step's does.  The structured
    # sweep needs no tensor (tens of MB).
    normals = torch.from_numpy(synth.make_map(w)).cuda()
    fac = g.init_factors_to_device(synth.init_factors(N, L, B, R, 2000 + w["seed"]))
    sws = g.CPWorkspace(N, L, B, R, "structured")
    sws.prepare(normal_xy=normals)
    sws.sweeps(fac, 1, report=False)
    del sws
    mat = g.QueryMaterial.from_factors(fac)
    g.build_query_tables(mat)
    qd = g.queries_to_device(synth.queries_fractional(N, L, B, nq, 1000 + w["seed"]))
    out = torch.empty(nq, dtype=torch.float32, device="cuda")
    status = g.new_status()
    qws = torch.empty(16, dtype=torch.uint8, device="cuda")
    grads = {k: torch.zeros_like(fac[a]) for k, a in
             (("dfx", "fx"), ("dfy", "fy"), ("dflw", "fl"), ("dfs", "fs"), ("dft", "ft"))}
    bws = torch.empty(g.backward_workspace_bytes(mat), dtype=torch.uint8, device="cuda")
    if args.query_tuning:
        tuning = tuple(int(v) for v in args.query_tuning.split(","))
    else:
        from paper_2109_14807_gb300 import tune
        tuning = tune.autotune_query(mat, qd, sample=2_000_000, repeats=2)

    def run():
        g.range_query(mat, qd, out=out, status=status, workspace=qws, tuning=tuning)
        g.range_query_backward(mat, qd, out, [grads], status=status, workspace=bws)

    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    lib.gsp_profile_reset()
    lib.gsp_profile_enable(1)
    for _ in range(args.steps):
        run()
    lib.gsp_profile_enable(0)
    rec = {}
    for pid in range(15):
        n_l, ms = _lib.c_int64(), _lib.c_double()
        _lib.check("gsp_profile_read", lib.gsp_profile_read(pid, n_l, ms))
        name = lib.gsp_profile_name(pid).decode()
        if n_l.value and name in QUERY_KERNELS:
            rec[name] = {"launches": n_l.value, "avg_launch_ms": ms.value / n_l.value,
                         "queries_per_s": nq / (ms.value / n_l.value / 1e3)}
    print(json.dumps({"metric": "query kernels alone (tables, range queries, adjoint)",
                      "workload": WORKLOAD, "N": N, "levels": L, "bins": B, "rank": R,
                      "queries": nq, "query_tuning": list(tuning), "kernels": rec,
                      "device_status": g.status_bits(status),
                      "device_gb": torch.cuda.max_memory_allocated() / 1e9}), flush=True)


# ------------------------------------------------------ precision report --
GOLDEN_FITS = os.path.join(ROOT, "tests", "golden", "brushed512_als_fits.txt")


def precision_report(args):
    """CP-ALS per MTTKRP precision: fit error after each of 20 sweeps against
    the FP64 oracle's fits from the same seeded init (stored by
    tests/golden/make_brushed512_fits.py), and the time of one sweep
    (CUDA events), on the 512^2 brushed map and on the benchmark map."""
    import numpy as np
    import torch
    import paper_2109_14807_gb300 as g
    torch.cuda.set_device(0)
    ref = np.loadtxt(GOLDEN_FITS, comments="#")[:, 1]
    out = {"metric": "CP-ALS fit error vs FP64 oracle and sweep time per MTTKRP precision",
           "data": "synthetic", "variants": {}}
    for wname in args.report_workloads.split(","):
        w = synth.WORKLOADS[wname]
        N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
        m = torch.from_numpy(synth.make_map(w)).cuda()
        init = synth.init_factors(N, L, B, R, 2000 + w["seed"])
        for prec in args.report_precisions.split(","):
            ws = g.CPWorkspace.for_map(L, B, R, prec, normal_xy=m)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ws.prepare(normal_xy=m)
            b.record()
            torch.cuda.synchronize()
            rec = out["variants"].setdefault(prec, {})
            prep_ms = a.elapsed_time(b)
            if wname == "brushed512" and prec == "structured_gaussian":
                # the Gaussian-footprint tensor is another tensor: its fit only
                f = g.init_factors_to_device(init)
                fits, _ = ws.sweeps(f, w["sweeps"])
                rec[wname] = {"final_fit": fits[-1], "footprint": "gaussian"}
            elif wname == "brushed512":
                f = g.init_factors_to_device(init)
                fits, _ = ws.sweeps(f, w["sweeps"])
                rel = np.abs(np.array(fits) - ref[: len(fits)]) / np.abs(ref[: len(fits)])
                rec[wname] = {"max_rel_fit_error": float(rel.max()), "final_fit": fits[-1]}
            else:
                rec[wname] = {}
            # sweep time: one untimed sweep, then 5 sweeps in one call (no host sync)
            f = g.init_factors_to_device(init)
            ws.sweeps(f, 1, report=False)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ws.sweeps(f, 5, report=False)
            b.record()
            torch.cuda.synchronize()
            rec[wname]["sweep_ms"] = round(a.elapsed_time(b) / 5, 3)
            rec[wname]["prepare_ms"] = round(prep_ms, 3)
            rec[wname]["workspace_mb"] = round(ws.buf.numel() / 2 ** 20, 1)
            if prec.startswith("structured"):
                rec[wname]["kernels"] = structured_kernels(ws, f, w)
            del ws
            torch.cuda.empty_cache()
    out["oracle_final_fit_brushed512"] = float(ref[-1])
    print(json.dumps(out), flush=True)


def structured_kernels(ws, f, w):
    """Per-sweep device time of the structured passes (library event pairs over
    5 sweeps) and their FP32 rate against the CUDA-core FMA peak: 152 SMs x 128
    FP32 lanes x 2 flops x the maximum SM clock.  Algorithmic flops per texel
    and rank: side pass 1 + 2L (h = fs * ft, then L FMAs), bin pass 2L + 2
    (L FMAs for P, one FMA into the bin table)."""
    from paper_2109_14807_gb300 import _lib
    lib = _lib.load()
    peaks, _ = load_peaks()
    alu_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    N, L, R = w["N"], w["levels"], w["rank"]
    lib.gsp_profile_reset()
    lib.gsp_profile_enable(1)
    ws.sweeps(f, 5, report=False)
    lib.gsp_profile_enable(0)
    flops = {"struct_side": N * N * R * (2 * L + 1), "struct_bins": N * N * R * (2 * L + 2)}
    out = {}
    for pid in range(15):
        n_l, ms = _lib.c_int64(), _lib.c_double()
        _lib.check("gsp_profile_read", lib.gsp_profile_read(pid, n_l, ms))
        name = lib.gsp_profile_name(pid).decode()
        if not n_l.value:
            continue
        rec = {"launches_per_sweep": n_l.value / 5, "ms_per_sweep": round(ms.value / 5, 4)}
        if name in flops:
            tf = flops[name] / (ms.value / n_l.value * 1e-3) / 1e12
            rec.update({"tflops": round(tf, 2), "alu_peak_tflops": round(alu_peak, 1),
                        "frac_of_alu_peak": round(tf / alu_peak, 3)})
        out[name] = rec
    return out


# ------------------------------------------------------- batching report --
BATCH_SHAPES = [(128, 16, 16), (128, 32, 64), (256, 16, 32), (256, 64, 32), (512, 32, 16),
                (512, 32, 64), (1024, 64, 32), (1024, 16, 64)]  # (N, rank, bins)


def batching_report(args):
    """Queries/s of one multi-material launch: 8 materials with seeded random
    factors, 5e7 camera-sweep queries (uneven footprint and angular size),
    the launch shape chosen by the autotuner on a 2e6-query sample, then the
    launch replayed from a CUDA graph (and, for comparison, launched eagerly)."""
    import numpy as np
    import torch
    import paper_2109_14807_gb300 as g
    from paper_2109_14807_gb300 import tune
    torch.cuda.set_device(0)
    mats = []
    for i, (N, R, B) in enumerate(BATCH_SHAPES):
        L = int(np.log2(N)) + 1
        fac = {}
        for j, (k, n) in enumerate((("fx", N), ("fy", N), ("fl", L), ("fs", B), ("ft", B))):
            fac[k] = torch.from_numpy((2 * synth.uniform(900 + i, j, n * R) - 1)
                                      .reshape(n, R).astype(np.float32)).cuda()
        fac["lambda"] = torch.from_numpy((0.5 + synth.uniform(900 + i, 9, R)).astype(np.float32)).cuda()
        mat = g.QueryMaterial.from_factors(fac)
        g.build_query_tables(mat)
        mats.append(mat)
    n = 50_000_000
    q = synth.queries_camera([(N, int(np.log2(N)) + 1, B) for N, R, B in BATCH_SHAPES], n, 2024)
    qd = g.queries_to_device(q)
    del q
    tn = tune.autotune_query(mats, qd, sample=2_000_000, repeats=2)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    graph = tune.QueryGraph(mats, qd, out, tuning=tn)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, args.steps // 3)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        graph.replay()
    b.record()
    torch.cuda.synchronize()
    ms_graph = a.elapsed_time(b) / reps
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    a.record()
    for _ in range(reps):
        g.range_query(mats, qd, out=out, tuning=tn, workspace=ws)
    b.record()
    torch.cuda.synchronize()
    ms_eager = a.elapsed_time(b) / reps
    print(json.dumps({"metric": "multi-material range queries/s (graph-captured, autotuned)",
                      "value": n / (ms_graph / 1e3), "unit": "queries/s", "ms_per_launch": ms_graph,
                      "eager_queries_per_s": n / (ms_eager / 1e3), "queries": n,
                      "materials": [{"N": N, "rank": R, "bins": B} for N, R, B in BATCH_SHAPES],
                      "tuning": {"lanes_per_query": tn[0], "blocks_per_sm": tn[1], "threads": tn[2],
                                 "chunk": tn[3]},
                      "data": "synthetic (seeded random factors, camera-sweep queries)"}), flush=True)


def sampling_report(args):
    """Samples/s of gsp_sample_ndf: 10^7 footprints (x, y, fractional level)
    of one 1024^2 material with 11 levels, 32^2 bins and rank 64 (seeded
    random non-negative factors), each descending log2(32) = 5 quad levels
    with four range queries per level."""
    import numpy as np
    import torch
    import paper_2109_14807_gb300 as g
    torch.cuda.set_device(0)
    N, L, B, R = 1024, 11, 32, 64
    fac = {}
    for j, (k, n) in enumerate((("fx", N), ("fy", N), ("fl", L), ("fs", B), ("ft", B))):
        fac[k] = torch.from_numpy(synth.uniform(950, j, n * R).reshape(n, R).astype(np.float32)).cuda()
    fac["lambda"] = torch.ones(R, dtype=torch.float32, device="cuda")
    mat = g.QueryMaterial.from_factors(fac)
    g.build_query_tables(mat)
    n = 10_000_000
    sd = g.samples_to_device(synth.sample_footprints(N, L, n, 951))
    ud = torch.from_numpy(synth.sample_uniforms(952, n)).cuda()
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        g.sample_ndf(mat, sd, ud, out=out)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, args.steps // 3)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        g.sample_ndf(mat, sd, ud, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    print(json.dumps({"metric": "hierarchical NDF importance samples/s (Sec. 5.2)",
                      "value": n / (ms / 1e3), "unit": "samples/s", "ms_per_launch": ms,
                      "samples": n, "range_queries_per_sample": 4 * 5,
                      "config": {"N": N, "levels": L, "bins": B, "rank": R},
                      "data": "synthetic (seeded random factors, uniform footprints)"}), flush=True)


def clustered_report(args):
    """The clustered compression layout of Sec. 4.2 (row f2) on a 256^2 flake
    map with 9 levels and 64^2 bins (16 angular blocks of 16^2 per image),
    rank 16: layout, batched per-group CP-ALS to |delta fit| < 1e-4 (at most
    500 sweeps, Sec. 4.2), compression ratio, and 10^6 fractional range queries
    through the block-splitting query kernel, with its HBM roofline."""
    import numpy as np
    import torch
    import paper_2109_14807_gb300 as g
    torch.cuda.set_device(0)
    wname = args.clustered_workload
    w = synth.WORKLOADS[wname]
    N, L, B, R = w["N"], w["levels"], w["bins"], w["rank"]
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    m = torch.from_numpy(synth.make_map(w)).cuda()
    H = g.build_footprint_ndfs(m, L, B)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    lay = g.cluster_layout(H)
    b.record()
    torch.cuda.synchronize()
    layout_ms = a.elapsed_time(b)
    off = lay["offsets"].cpu().numpy()
    init = synth.cluster_init(lay["G"], off, R, 6006)
    st = g.new_status()
    a, b = ev(), ev()
    a.record()
    fac = g.cluster_decompose(H, lay, R, init, max_sweeps=500, tol=1e-4, status=st)
    b.record()
    torch.cuda.synchronize()
    als_ms = a.elapsed_time(b)
    sweeps = fac["sweeps"].cpu().numpy()
    fits = fac["fit"].cpu().numpy()
    nonempty = np.diff(off) > 0
    t = g.CLUSTER_BLOCK
    stored = int(sum(R * (2 * t + int(mj) + 1) + 2 * R * (t + 1) for mj in np.diff(off) if mj))
    ratio = stored / float(L * N * N * B * B)
    tab = g.cluster_tables(lay, fac)
    q = synth.queries_fractional(N, L, B, w["queries"], 6007, frac_level=True)
    qd = g.queries_to_device(q)
    out = torch.empty(len(q), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, args.warmup)):
        g.cluster_range_query(lay, tab, qd, out=out)
    times = []
    for _ in range(max(3, args.steps // 3)):
        flush.zero_()  # L2 flush between timed launches
        a, b = ev(), ev()
        a.record()
        g.cluster_range_query(lay, tab, qd, out=out)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    qms = float(np.median(times))
    # algorithmic bytes per query: the descriptor, then for each of the two
    # blended levels one z-map word, the group offset and, per rank, two SAT
    # rows of each in-block factor and one Z row entry (blocks crossed: 1 for
    # almost every range of the mix)
    per_q = 32 + 2 * (8 + R * (2 * 16 + 2 * 16 + 4))
    peaks, src = load_peaks()
    peak = float(peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    achieved = per_q * len(q) / (qms / 1e3) / 1e9
    print(json.dumps({
        "metric": "clustered layout (Sec. 4.2): per-group CP-ALS and block-splitting range queries",
        "config": {"workload": wname, "N": N, "levels": L, "bins": B, "block": t, "region": 8,
                   "rank": R, "groups": lay["G"], "queries": len(q)},
        "layout_ms": layout_ms, "members": lay["total"], "largest_group": lay["max_members"],
        "nonempty_groups": int(nonempty.sum()),
        "blank_blocks_dropped": 1.0 - lay["total"] / float(L * N * N * (B // t) ** 2),
        "als_ms": als_ms, "als_sweeps_mean": float(sweeps[nonempty].mean()),
        "als_sweeps_max": int(sweeps.max()), "fit_min": float(fits[nonempty].min()),
        "fit_median": float(np.median(fits[nonempty])), "status": g.status_bits(st),
        "compression_ratio": ratio,
        "query_ms": qms, "queries_per_s": len(q) / (qms / 1e3),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "bytes_per_query": per_q,
                     "peak_source": src},
        "data": "synthetic (seeded flake map, seeded initial factors)"}), flush=True)


def env_report(args):
    """Environment-light prefiltering (Sec. 5.4, row f4): gsp_env_queries turns
    10^7 shading records (footprint, outgoing direction, SG lobe) against 64
    spherical-Gaussian lobes into range-query descriptors of one 1024^2 material
    (11 levels, 32^2 bins, rank 64, seeded random non-negative factors), which
    gsp_range_query answers (launch shape from the autotuner, or --query-tuning);
    both launches timed with CUDA events."""
    import numpy as np
    import torch
    import paper_2109_14807_gb300 as g
    torch.cuda.set_device(0)
    N, L, B, R = 1024, 11, 32, 64
    fac = {}
    for j, (k, n) in enumerate((("fx", N), ("fy", N), ("fl", L), ("fs", B), ("ft", B))):
        fac[k] = torch.from_numpy(synth.uniform(960, j, n * R).reshape(n, R).astype(np.float32)).cuda()
    fac["lambda"] = torch.ones(R, dtype=torch.float32, device="cuda")
    mat = g.QueryMaterial.from_factors(fac)
    g.build_query_tables(mat)
    n, n_sg = 10_000_000, 64
    sgs = torch.from_numpy(synth.env_lobes(n_sg, 961).view(np.float32).reshape(n_sg, 8)).cuda()
    rec = torch.from_numpy(synth.env_records([(N, L, B)], n, n_sg, 962).view(np.int32).reshape(n, 8)).cuda()
    qd = torch.empty((n, 8), dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    g.env_queries(mat, sgs, rec, out=qd)
    if args.query_tuning:
        tuning = tuple(int(v) for v in args.query_tuning.split(","))
    else:
        from paper_2109_14807_gb300 import tune
        tuning = tune.autotune_query(mat, qd, sample=2_000_000, repeats=2)
    for _ in range(max(3, args.warmup)):
        g.env_queries(mat, sgs, rec, out=qd)
        g.range_query(mat, qd, out=out, tuning=tuning)
    gen, qry = [], []
    for _ in range(max(3, args.steps // 3)):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record()
        g.env_queries(mat, sgs, rec, out=qd)
        b.record()
        g.range_query(mat, qd, out=out, tuning=tuning)
        c.record()
        torch.cuda.synchronize()
        gen.append(a.elapsed_time(b))
        qry.append(b.elapsed_time(c))
    gms, qms = float(np.median(gen)), float(np.median(qry))
    # the generator streams 32-byte records and SG lobes in and 32-byte
    # descriptors out: 64 bytes per record
    peaks, src = load_peaks()
    peak = float(peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    achieved = 64.0 * n / (gms / 1e3) / 1e9
    print(json.dumps({
        "metric": "environment-light prefiltering (Sec. 5.4): records/s through descriptor generation and range query",
        "value": n / ((gms + qms) / 1e3), "unit": "records/s", "records": n, "sg_lobes": n_sg,
        "generator_ms": gms, "range_query_ms": qms, "query_tuning": list(tuning),
        "generator_roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": achieved / peak, "bytes_per_record": 64, "peak_source": src},
        "config": {"N": N, "levels": L, "bins": B, "rank": R},
        "data": "synthetic (seeded random factors, lobes and records)"}), flush=True)


def main():
    args = parse_args()
    if args.query_profile:
        query_profile(args)
        return
    if args.env_report:
        env_report(args)
        return
    if args.clustered_report:
        clustered_report(args)
        return
    if args.sampling_report:
        sampling_report(args)
        return
    if args.batching_report:
        batching_report(args)
        return
    if args.precision_report:
        precision_report(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    try:
        run_gsp(args, rank, world)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
