"""Host-side logic of the measurement scripts: roofline arithmetic, the
committed ncu traffic lookup, workload descriptions, sections and row samples."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1112_0059_gb300 import synth  # noqa: E402


def test_scan_roofline_arithmetic():
    prof = {"search_ms": 2000.0, "search_launches": 2}
    peaks = {"bf16_tflops_sustained": 1000.0}
    r = bench.scan_roofline(prof, 1_000_000, 500_000, peaks, "measured", True, None)
    flops = 2.0 * 128 * 1_000_000 * 500_000
    assert r["flops_per_launch"] == flops and r["avg_launch_ms"] == 1000.0
    assert abs(r["achieved"] - flops / 1.0 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["kernel"] == "tc_scan_kernel<FmtBf16, KnnEpilogue<16>, 1, 0>"
    f = bench.scan_roofline(prof, 1_000_000, 500_000, peaks, "measured", True, 32, plan={"tile_m": 256})
    assert f["peak"] == 2000.0 and f["kernel"] == "tc_scan_kernel<FmtE4m3, KnnEpilogue<32>, 2, 0>"
    assert bench.scan_roofline(prof, 10, 10, peaks, "x", True, 24)["kernel"].endswith("KnnEpilogue<24>, 1, 0>")
    smem = {"tile_m": 128, "list_storage": "shared memory"}
    assert bench.scan_roofline(prof, 10, 10, peaks, "x", True, 64, plan=smem)["kernel"].endswith("KnnSmemEpilogue<64>, 1, 0>")
    assert bench.scan_roofline(prof, 10, 10, peaks, "x", True, 128)["kernel"].endswith("KnnEpilogue<0>, 1, 0>")
    assert bench.scan_roofline(prof, 10, 10, peaks, "x", True, None, 20)["kernel"].endswith("<FmtBf16, KnnEpilogue<24>, 1, 0>")
    assert bench.scan_roofline(prof, 10, 10, peaks, "x", True, None, 100)["kernel"].endswith("<FmtBf16, KnnEpilogue<0>, 1, 0>")
    assert bench.scan_roofline(prof, 10, 10, peaks, "x", False, None)["kernel"].endswith("NbnnEpilogue, 1, 0>")
    chunk = {"tile_m": 128, "chunked": 1}  # the claimed-chunk instantiation
    assert bench.scan_roofline(prof, 10, 10, peaks, "x", True, 24, plan=chunk)["kernel"].endswith("KnnEpilogue<24>, 1, 1>")


def test_traffic_lookup_matches_committed_capture():
    with open(bench.TRAFFIC_FILE) as f:
        t = json.load(f)
    name = "tc_scan_kernel<FmtBf16, KnnEpilogue<16>, 1, 0>"
    k = t["kernels"][name]
    got = bench.traffic_per_launch(name, k["query_rows"], k["n_ref"])
    if t["kernel_hash"] == bench.kernel_hash():
        assert got == pytest.approx(k["dram_bytes"])
        # scaled by query rows x references
        assert bench.traffic_per_launch(name, 2 * k["query_rows"], 3 * k["n_ref"]) == pytest.approx(6 * got)
    else:  # sources changed since the capture: no stale number is reported
        assert got is None
    assert bench.traffic_per_launch("no such kernel", 750000, 11520000) is None
    assert bench.traffic_note("no such kernel", 750000, 11520000).startswith("no ncu capture")
    if t["kernel_hash"] == bench.kernel_hash():
        # the capture's own size: its figure as measured; another size: scaled
        assert "this launch" in bench.traffic_note(name, k["query_rows"], k["n_ref"])
        assert "scaled" in bench.traffic_note(name, k["query_rows"] // 2, k["n_ref"])


def test_measured_peaks_and_workload_config():
    peaks, src = bench.measured_peaks()
    assert src in ("measured", "fallback") and peaks["bf16_tflops_sustained"] > 0
    cfg = bench.workload_config(synth.workload("caltech256-like"), 10)
    assert cfg["n_ref"] == 11_520_000 and cfg["query_descriptors"] == 750_000 and cfg["k"] == 10
    assert "larger than L2" in cfg["l2"]
    assert bench.workload_config(synth.workload("tiny"), 10, "nbnn")["k"] is None


def test_roofline_clock_normalised():
    prof = {"search_ms": 1000.0, "search_launches": 1, "search_cycles_per_tile": 1280.0, "search_sm_clock_ghz": 1.9}
    peaks = {"bf16_tflops_sustained": 1000.0, "clocks_under_load": {"sm_mhz_median": 1470.0}}
    r = bench.scan_roofline(prof, 10, 10, peaks, "measured", True, None)
    assert r["mma_floor_cycles_per_tile"] == 1152 and r["tensor_pipe_frac_at_kernel_clock"] == 1152 / 1280
    assert abs(r["algorithmic_frac_at_kernel_clock"] - 0.8) < 1e-12 and r["peak_sm_mhz"] == 1470.0
    f = bench.scan_roofline(prof, 10, 10, peaks, "measured", True, 32)
    assert f["mma_floor_cycles_per_tile"] == 640 and abs(f["algorithmic_frac_at_kernel_clock"] - 0.4) < 1e-12
    assert "cycles_per_tile" not in bench.scan_roofline({"search_ms": 1.0, "search_launches": 1}, 10, 10, peaks,
                                                        "measured", True, None)


def test_sections_and_row_samples():
    assert set(bench.DEFAULT_SECTIONS.split(",")) <= set(bench.SECTIONS)
    r = bench._sample(1000, 100, 7)
    assert len(r) == 100 and len(set(r.tolist())) == 100 and (r[1:] > r[:-1]).all() and r.max() < 1000
    assert bench._sample(50, 100, 7).tolist() == list(range(50))
    assert bench._sample(1000, 100, 7).tolist() == r.tolist()  # seeded
