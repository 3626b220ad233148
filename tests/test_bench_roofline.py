"""bench.py's roofline object for the dominant kernel of the step: the
tensor-core product launches count the six BF16 partial products of the
three-way split per FP32 multiply-add against the sustained BF16 peak, the
CUDA-core tiles count FP32 FMAs against the derived FFMA peak, vector
kernels are HBM bound.  Pure host arithmetic, checked on the CPU."""
import pytest

import bench

STATS = {"near_entries": 16_000_000, "far_u_entries": 28_000_000, "far_v_entries": 27_000_000,
         "aca_entries": 64_000_000}
NC = 65
SMS = 152


def test_tensor_core_row_launch_counts_six_bf16_products_against_the_sustained_peak():
    st = dict(STATS, product_path=1)
    avg_ms = 0.172
    r = bench.roofline({"hmm_rows": (60, 60 * avg_ms), "gmres_dots": (60, 1.0)}, st, 5, NC, SMS)
    flops = 6 * 2.0 * NC * (st["near_entries"] + st["far_u_entries"])
    assert r["kernel"] == "hmm_rows" and r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(flops / (avg_ms * 1e-3) / 1e12)
    assert r["peak"] == pytest.approx(bench.load_bf16_peak()[0])
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # DRAM traffic of the tensor-core row launch from its capture
    assert r["traffic"] == bench.TRAFFIC[(bench.workload_key(), "hmm_rows", 1)]


def test_tensor_core_far_launch_counts_the_v_panels():
    st = dict(STATS, product_path=1)
    r = bench.roofline({"hmm_far_vt": (12, 12 * 0.145)}, st, 1, NC, SMS)
    assert r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(6 * 2.0 * NC * st["far_v_entries"] / 0.145e-3 / 1e12)


def test_cuda_core_tiles_count_fp32_fmas_against_the_derived_peak():
    st = dict(STATS, product_path=0)
    avg_ms = 0.268
    r = bench.roofline({"hmm_rows": (60, 60 * avg_ms)}, st, 5, NC, SMS)
    smax = bench.load_peaks()[1]
    assert r["bound"] == "alu"
    assert r["peak"] == pytest.approx(SMS * 128 * 2 * smax * 1e6 / 1e12)
    assert r["achieved"] == pytest.approx(2.0 * NC * (st["near_entries"] + st["far_u_entries"]) / (avg_ms * 1e-3) / 1e12)
    # no capture of the current CUDA-core kernel: traffic unknown
    assert r["traffic"] is None


def test_vector_kernels_are_hbm_bound():
    r = bench.roofline({"gmres_cgs_update": (36, 5.0)}, dict(STATS, product_path=1), 1, NC, SMS)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["peak"] == pytest.approx(bench.load_peaks()[0])
