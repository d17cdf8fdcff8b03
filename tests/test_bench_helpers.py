"""Host-side arithmetic of bench.py (roofline entry, traffic lookup), on made-up timings."""
import json

import bench
from synth import CONFIGS


def _st(scan, resc, assign):
    return {"scan_kernel_ms": scan, "rescore_kernel_ms": resc, "assign_kernel_ms": assign}


def test_roofline_picks_dominant_kernel_and_its_roof():
    cfg = CONFIGS["db12000x64_d4096_k1024"]
    peaks = {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0}
    pairs, D = 7.3e8, cfg.dim
    # rescore dominant and compute-bound: 6 * pairs * D flops in 12 ms
    r = bench.roofline(cfg, _st(3.0, 12.0, 1.0), pairs, 6e9, 12e9, 64000, peaks, "measured")
    assert r["kernel"] == "rescore" and r["bound"] == "tensor"
    assert abs(r["achieved"] - 6 * pairs * D / 12e-3 / 1e12) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 2000.0) < 1e-12
    assert r["unit"] == "TFLOP/s" and json.dumps(r)
    # the same kernel reading 210 GB in 31 ms is HBM-bound
    r = bench.roofline(CONFIGS["db200000x64_d4096_k4096_fp8"], _st(8.0, 31.0, 1.2), 7.3e8, 47e9, 210e9, 16384,
                       peaks, "measured", with_traffic=False)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None
    assert abs(r["achieved"] - 210e9 / 31e-3 / 1e9) < 1e-6 * r["achieved"]
    # the FP8 scan is held against twice the BF16 peak
    assert r["all"]["scan"].get("tensor_frac") is not None


def test_recorded_traffic_ignores_other_sources(tmp_path, monkeypatch):
    assert bench.recorded_traffic("no-such-kernel", "0" * 12) == (None, None, None)


def test_roofline_without_tensor_core_scan():
    """An FP32 store scans on the CUDA cores: no scan or rescore kernel time, only the quantiser."""
    cfg = CONFIGS["db200x64_d128_k64"]
    r = bench.roofline(cfg, _st(0.0, 0.0, 0.05), 1e6, 1e8, 0, 640, {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0},
                       "measured")
    assert r["kernel"] == "quantiser" and r["scan_hbm"]["achieved_gbs"] is None
    assert bench.roofline(cfg, _st(0.0, 0.0, 0.0), 0, 0, 0, 0, {"hbm_gbs": 1.0, "bf16_tflops": 1.0}, "m") is None


def test_roofline_names_the_fused_pass():
    """A BF16 store with rescore rows runs scan and rescore as one kernel: no scan time of its own,
    the entry is the fused kernel with the three-product FLOPs over every scanned pair."""
    cfg = CONFIGS["db12000x64_d4096_k1024"]
    peaks = {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0}
    pairs = 7.46e8
    r = bench.roofline(cfg, _st(0.0, 12.35, 0.97), pairs, 6e9, 12.5e9, 64000, peaks, "measured", with_traffic=False)
    assert r["kernel"] == "fused scan + rescore" and r["bound"] == "tensor"
    assert abs(r["achieved"] - 6 * pairs * cfg.dim / 12.35e-3 / 1e12) < 1e-6 * r["achieved"]
    assert "scan" not in r["all"] and "rescore" not in r["all"]
    # an FP8 store keeps the separate scan and rescore
    r = bench.roofline(CONFIGS["db200000x64_d4096_k4096_fp8"], _st(8.1, 32.0, 1.0), pairs, 47e9, 188e9, 32768,
                       peaks, "measured", with_traffic=False)
    assert r["kernel"] == "rescore" and "scan" in r["all"]


def test_roofline_counts_the_rescore_candidates():
    """With the candidate counters the separate rescore's work is its candidate pairs and rows;
    the fused pass keeps its three-product accounting and reports the method's work beside it."""
    peaks = {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0}
    cfg = CONFIGS["db200000x64_d4096_k4096_fp8"]
    cand = {"rescore_items": 1000, "rescore_items_kept": 400, "cand_pairs": 2e8, "cand_rows": 5e6,
            "rescore_rows_read": 5.1e6}
    r = bench.roofline(cfg, _st(8.0, 14.0, 1.0), 7.3e8, 47e9, 188e9, 32768, peaks, "measured", with_traffic=False,
                       cand=cand)
    assert r["kernel"] == "rescore" and r["bound"] == "hbm"
    assert abs(r["achieved"] - 5e6 * (4 * cfg.dim + 12) / 14e-3 / 1e9) < 1e-6 * r["achieved"]
    assert r["candidate_work"]["items_kept_fraction"] == 0.4
    c2 = CONFIGS["db12000x64_d4096_k1024"]
    r = bench.roofline(c2, _st(0.0, 12.0, 1.0), 7.3e8, 6e9, 12e9, 64000, peaks, "measured", with_traffic=False,
                       cand=dict(cand, cand_pairs=1e8))
    assert r["kernel"] == "fused scan + rescore"
    assert abs(r["achieved"] - 6 * 7.3e8 * c2.dim / 12e-3 / 1e12) < 1e-6 * r["achieved"]
    m = (2 * 7.3e8 + 6 * 1e8) * c2.dim / 12e-3 / 1e12 / 2000.0
    assert abs(r["candidate_work"]["method_work_frac"] - m) < 1e-9


def test_traffic_is_scaled_by_the_launch_units(tmp_path, monkeypatch):
    """A capture on a reduced case gives bytes per unit; the entry's traffic is that times the
    units the timed launch processed (here rows the rescore read)."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.md").write_text(
        "| kernel | source hash | capture | bytes per unit | unit | note |\n"
        "|---|---|---|---|---|---|\n"
        "| rescore | abc123 | reduced | 16500 | rescore row read | x |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda files: "abc123")
    cand = {"rescore_items": 10, "rescore_items_kept": 9, "cand_pairs": 1e8, "cand_rows": 9e6,
            "rescore_rows_read": 1.1e7}
    r = bench.roofline(CONFIGS["db200000x64_d4096_k4096_fp8"], _st(8.0, 31.0, 1.0), 7e8, 47e9, 188e9, 32768,
                       {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0}, "measured", cand=cand)
    assert r["kernel"] == "rescore"
    assert r["traffic"] == 16500 * 1.1e7 and "reduced" in r["traffic_source"]
    monkeypatch.setattr(bench, "kernel_source_hash", lambda files: "changed")
    r = bench.roofline(CONFIGS["db200000x64_d4096_k4096_fp8"], _st(8.0, 31.0, 1.0), 7e8, 47e9, 188e9, 32768,
                       {"hbm_gbs": 7000.0, "bf16_tflops": 2000.0}, "measured", cand=cand)
    assert r["traffic"] is None
