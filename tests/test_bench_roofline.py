"""Host arithmetic of bench.py's JSON line, checked without a GPU: the roofline records
(achieved = algorithmic work over device time, the peak each family is held against, the
DRAM traffic scaled from the captured bytes per block), the replica value and seeds, and
the peaks file fallback."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6772.0, "bf16_tflops": 1962.0, "bf16_tflops_sustained": 1723.0,
         "sm_max_mhz": 2070.0}


def test_invert_record_counts_flops_against_the_tensor_rate():
    ny, blocks, steps = 160, 2020, 20
    flops = 8.0 * ny ** 3 * blocks * steps            # complex Gauss-Jordan: 8 n^3 per block
    ms = 3.3 * steps
    r = bench._roofline("invert", {"ms": ms, "flops": flops, "bytes": 0.0, "steps": steps},
                        1, PEAKS, "measured", ny=ny, live={"tf32_tcgen05_tflops": 1200.0})
    achieved = 3 * flops / (ms * 1e-3) / 1e12         # 3xTF32 tensor products
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s" and r["kernel"] == "invert"
    assert r["achieved"] == pytest.approx(achieved, abs=1e-3)
    assert r["peak"] == 1200.0
    assert r["frac"] == pytest.approx(achieved / 1200.0, abs=1e-4)
    if bench.GJ_TC_DRAM_BYTES_PER_BLOCK_NY160:
        assert r["traffic"] == round(bench.GJ_TC_DRAM_BYTES_PER_BLOCK_NY160 * blocks)
        # each block is read once and its inverse written once
        assert 8 * ny * ny <= bench.GJ_TC_DRAM_BYTES_PER_BLOCK_NY160 <= 2 * 8 * ny * ny * 1.01
    else:
        assert r["traffic"] is None


def test_fp64_invert_record_is_held_against_the_fp64_rate():
    stats = {"ms": 10.0, "flops": 8.0 * 96 ** 3 * 10, "bytes": 0.0, "steps": 1}
    r = bench._roofline("invert", stats, 0, PEAKS, "measured", ny=160,
                        live={"fp64_fma_tflops": 1.05})
    assert r["bound"] == "alu" and r["peak"] == 1.05 and r["traffic"] is None


def test_fp32_gemm_record_is_held_against_the_tf32_tensor_rate():
    flops = 1.0e12
    r = bench._roofline("gemm", {"ms": 10.0, "flops": flops, "bytes": 0.0}, 1, PEAKS, "measured")
    assert r["bound"] == "tensor"
    # three TF32 products per complex product (3xTF32)
    assert r["achieved"] == pytest.approx(3 * flops / 1e-2 / 1e12, abs=1e-3)
    assert r["peak"] == pytest.approx(1723.0 * 1.1 / 2.25, abs=0.1)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)


def test_fp64_families_use_the_nominal_fp64_rate():
    r = bench._roofline("gemm", {"ms": 1.0, "flops": 1e9, "bytes": 0.0}, 0, PEAKS, "measured")
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_NOMINAL_TFLOPS


def test_streaming_family_is_held_against_measured_hbm():
    r = bench._roofline("solve", {"ms": 2.0, "flops": 0.0, "bytes": 7.2e9}, 1, PEAKS, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(7.2e9 / 2e-3 / 1e9, abs=0.1)
    assert r["peak"] == 6772.0
    assert r["frac"] == pytest.approx(r["achieved"] / 6772.0, abs=1e-4)


def test_no_record_without_device_time():
    assert bench._roofline("solve", {"ms": 0.0, "flops": 0.0, "bytes": 1.0}, 1, PEAKS, "x") is None


def test_replica_value_and_disjoint_seeds():
    assert bench._replica_value(4, 100, 2000.0) == pytest.approx(200.0)
    seeds = [set(bench._replica_seeds(r, 64)) for r in range(8)]
    for i in range(8):
        assert len(seeds[i]) == 64
        for j in range(i):
            assert not seeds[i] & seeds[j]


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench._peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.0}))
    peaks, kind = bench._peaks()
    assert kind == "measured" and peaks["hbm_gbs"] == 7000.0


def test_measured_peaks_of_the_run_replace_the_derived_ones():
    live = {"fp32_fma_tflops": 70.0, "fp64_fma_tflops": 1.1, "tf32_tcgen05_tflops": 1000.0}
    st = {"ms": 10.0, "flops": 1.0e12, "bytes": 0.0, "steps": 1}
    g = bench._roofline("gemm", st, 1, PEAKS, "measured", live=live)
    assert g["peak"] == 1000.0 and "measured in this run" in g["peak_source"]
    assert g["frac"] == pytest.approx(300.0 / 1000.0, rel=1e-3)
    inv = bench._roofline("invert", st, 1, PEAKS, "measured", ny=96, live=live)
    assert inv["peak"] == 1000.0 and inv["bound"] == "tensor"
    lvl = bench._roofline("level0", st, 1, PEAKS, "measured", live=live)
    assert lvl["peak"] == 70.0 and lvl["frac"] == pytest.approx(100.0 / 70.0, rel=1e-3)
    g64 = bench._roofline("gemm", st, 0, PEAKS, "measured", live=live)
    assert g64["peak"] == 1.1
    q = bench._roofline("qform", st, 1, PEAKS, "measured", live=live)
    assert q["peak"] == 1.1 and q["bound"] == "alu"
