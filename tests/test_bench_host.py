"""Host logic of bench.py that needs no GPU: the roofline of the kernel with
the largest share of the step, the algorithmic bytes per launch it uses, and
the per-launch DRAM traffic read from the committed ncu summary."""
import bench


W = {"N": 1024, "levels": 11, "bins": 32, "rank": 64, "queries": 10_000_000}
PEAKS = {"hbm_gbs": 6793.4}


def _prof(**ms):
    # kernel -> (launches, total ms), one launch each
    return {k: (1, v) for k, v in ms.items()}


def test_roofline_reports_the_largest_share_with_algorithmic_bytes():
    prof = _prof(box_hist=1.1, mttkrp_xy=0.46, mttkrp_lst=0.46, range_query=1.7,
                 range_query_backward=3.2, solve=0.15)
    r = bench.roofline(prof, W, "bf16", PEAKS, "measured", 67, 80)
    assert r["kernel"] == "range_query_backward"
    per_query = 2 * 11 * 64 * 4 + 36
    assert r["algorithmic_bytes_per_launch"] == W["queries"] * per_query
    assert abs(r["achieved"] - W["queries"] * per_query / 3.2e-3 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / PEAKS["hbm_gbs"]) < 1e-12
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and "note" in r
    assert (r["occupied_bins"], r["operand_columns"]) == (67, 80)
    # the others, by share, with the operand kernels' bytes from the stored columns
    names = [o["kernel"] for o in r["others"]]
    assert names[0] == "range_query" and set(names) == {"range_query", "box_hist", "mttkrp_xy", "mttkrp_lst"}
    x = 1024 * 1024 * 11 * 80
    box = next(o for o in r["others"] if o["kernel"] == "box_hist")
    assert abs(box["achieved"] - x * 2 / 1.1e-3 / 1e9) < 1e-6 * box["achieved"]
    xy = next(o for o in r["others"] if o["kernel"] == "mttkrp_xy")
    assert abs(xy["achieved"] - (x * 2 + 1024 * 1024 * 64 * 4) / 0.46e-3 / 1e9) < 1e-6 * xy["achieved"]


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
