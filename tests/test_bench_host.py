"""Host logic of bench.py that needs no GPU: the roofline of the kernel with
the largest share of the step, the algorithmic bytes per launch it uses, and
the per-launch DRAM traffic read from the committed ncu summary."""
import bench


W = {"N": 1024, "levels": 11, "bins": 32, "rank": 64, "queries": 10_000_000}
PEAKS = {"hbm_gbs": 6793.4}


def _prof(**ms):
    # kernel -> (launches, total ms), one launch each
    return {k: (1, v) for k, v in ms.items()}


def test_roofline_reports_the_largest_share_with_algorithmic_bytes(monkeypatch, tmp_path):
    # the query kernels are bound by the L1 data pipe: L1 wavefronts counted by
    # ncu for the same code and launch shape x 128 B over the live launch time,
    # against one wavefront per clock per SM; the gather bytes of the query
    # definition stay beside it as a ratio to the HBM peak
    h = bench._src_hash(("query.cu",))
    f = tmp_path / "onchip.txt"
    f.write_text("# kernel workload lanes wavefronts hash\n"
                 f"range_query_backward {bench.WORKLOAD} auto 300000000 {h}\n"
                 f"range_query {bench.WORKLOAD} 8 320000000 {h}\n")
    monkeypatch.setattr(bench, "ONCHIP_FILE", str(f))
    prof = _prof(box_hist=1.1, mttkrp_xy=0.46, mttkrp_lst=0.46, range_query=1.7,
                 range_query_backward=3.2, solve=0.15)
    r = bench.roofline(prof, W, "bf16", PEAKS, "measured", 67, 80, n_sm=152, sm_mhz=2000.0,
                       lanes={"range_query": 8, "range_query_backward": "auto"})
    assert r["kernel"] == "range_query_backward"
    assert r["bound"] == "l1" and r["unit"] == "GB/s"
    assert r["l1_wavefronts_per_launch"] == 300000000
    assert abs(r["achieved"] - 300000000 * 128 / 3.2e-3 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["peak"] - 152 * 128 * 2000e6 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    per_query = 2 * 11 * 64 * 4 + 36
    assert r["gather_bytes_per_launch"] == W["queries"] * per_query
    assert abs(r["gather_vs_hbm_peak"] - W["queries"] * per_query / 3.2e-3 / 1e9 / PEAKS["hbm_gbs"]) < 1e-9
    assert (r["occupied_bins"], r["operand_columns"]) == (67, 80)
    # the others, by share, with the operand kernels' bytes from the stored columns
    names = [o["kernel"] for o in r["others"]]
    assert names[0] == "range_query" and set(names) == {"range_query", "box_hist", "mttkrp_xy", "mttkrp_lst"}
    fwd = r["others"][0]
    assert fwd["bound"] == "l1" and abs(fwd["achieved"] - 320000000 * 128 / 1.7e-3 / 1e9) < 1e-3
    x = 1024 * 1024 * 11 * 80
    box = next(o for o in r["others"] if o["kernel"] == "box_hist")
    assert box["bound"] == "hbm"
    assert abs(box["achieved"] - x * 2 / 1.1e-3 / 1e9) < 1e-3
    xy = next(o for o in r["others"] if o["kernel"] == "mttkrp_xy")
    assert abs(xy["achieved"] - (x * 2 + 1024 * 1024 * 64 * 4) / 0.46e-3 / 1e9) < 1e-3
    # counters of another launch shape, or of changed code, are not used
    r2 = bench.roofline(prof, W, "bf16", PEAKS, "measured", 67, 80,
                        lanes={"range_query": 16, "range_query_backward": "auto"})
    assert r2["others"][0]["achieved"] is None and r2["others"][0]["frac"] is None
    f.write_text(f"range_query_backward {bench.WORKLOAD} auto 300000000 000000000000\n")
    r3 = bench.roofline(prof, W, "bf16", PEAKS, "measured", 67, 80)
    assert r3["l1_wavefronts_per_launch"] is None and r3["frac"] is None


def test_roofline_of_an_unmodelled_top_kernel_is_absent():
    assert bench.roofline(_prof(solve=5.0, box_hist=1.0), W, "bf16", PEAKS, "measured", 67, 80) is None
    assert bench.roofline({}, W, "bf16", PEAKS, "measured", 67, 80) is None


def test_traffic_rows_follow_the_source_hashes(monkeypatch, tmp_path):
    h = bench._src_hash(bench.KERNEL_SOURCE["range_query"])
    f = tmp_path / "traffic.txt"
    f.write_text("# kernel workload precision bytes hash\n"
                 f"range_query {bench.WORKLOAD} bf16 350000000 {h}\n"
                 f"box_hist {bench.WORKLOAD} bf16 1800000000 000000000000\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.ncu_traffic("range_query", "bf16") == 350000000.0
    assert bench.ncu_traffic("range_query", "fp32") is None      # no row for that precision
    assert bench.ncu_traffic("box_hist", "bf16") is None         # the source changed since
    assert bench.ncu_traffic("solve", "bf16") is None            # not a modelled kernel
