"""bench.py's roofline arithmetic (SURVEY 8(d) units), on CPU: the algorithmic
bytes of an expansion, the slower of the HBM / FP32 / SFU bounds, and the
measured DRAM traffic read from a committed ncu summary only while the kernel
sources are those it was captured from."""
import os

import pytest

import bench


def test_algorithmic_bytes():
    ab = bench.algo_bytes(n_tags=10, n_words=40, n_styles=2, n_paths=3, n_prims=100, arcs=False)
    assert ab["input"] == 10 + 160 + 48
    assert ab["scan_soa"] == 2 * 17 * 10
    assert ab["outline"] == 2000 and bench.algo_bytes(10, 40, 2, 3, 100, True)["outline"] == 2400
    assert ab["offsets"] == 8 * 11 + 8 * 4
    assert ab["total"] == ab["input"] + ab["scan_soa"] + ab["outline"] + ab["offsets"]
    assert ab["stages"]["emit"] == 2000 and ab["stages"]["tag_scan"] == 10 + 170


def test_roofline_takes_the_slower_bound():
    # 1 GB at 1000 GB/s = 1 ms; 40.27e9 FP32 instr at 152 x 128 x 2070 MHz = 1 s
    r = bench.roofline_of(1e9, 0, 0, 10.0, 1000.0, 152, 2070.0)
    assert r["bound"] == "hbm" and abs(r["frac"] - 0.1) < 1e-12 and abs(r["achieved"] - 100.0) < 1e-9
    fp32_peak, sfu_peak = bench.alu_peaks(152, 2070.0)
    assert abs(fp32_peak - 152 * 128 * 2.07e9) < 1 and abs(sfu_peak - 152 * 16 * 2.07e9) < 1
    verts = fp32_peak / bench.VERT_FP32 * 2e-3      # 2 ms of FP32 work
    r = bench.roofline_of(1e6, 0, verts, 4.0, 1000.0, 152, 2070.0)
    assert r["bound"] == "alu" and abs(r["frac"] - 0.5) < 1e-9
    assert abs(r["time_at_bounds_ms"]["fp32"] - 2.0) < 1e-9


def test_traffic_needs_the_captured_sources(tmp_path, monkeypatch):
    prof = os.path.join(bench.ROOT, "profiles")
    name = "_test_traffic_probe.md"
    path = os.path.join(prof, name)
    try:
        with open(path, "w") as f:
            f.write("traffic-per-unit: 12.5 bytes per primitive, sources 0000000000000000\n")
        assert bench.traffic_from_profiles(name, 1000) is None        # sources changed since
    finally:
        os.remove(path)
    assert bench.traffic_from_profiles("no_such_file.md", 10) is None
