"""The bench line's roofline arithmetic on fixed inputs (CPU): the dominant
kernel, achieved = algorithmic work per launch / mean launch time, the peak
derived from unit counts and the maximum SM clock, the fraction, the traffic
guard on the profiled source, and the end-to-end FP32 roofline."""
import hashlib
import os

import pytest

import bench

PK = {"sm_max_mhz": 2070.0, "hbm_gbs": 6785.9}
WORK = {"energy_pairs": 1000, "energy_modes": 40000, "lm_pairs": 3000, "lm_modes": 120000,
        "lm_inliers": 2000, "lm_trial": 1500, "rays": 10_000_000, "icp_pixels": 0,
        "hyp_attempts": 5_000_000, "hyp_stage2": 400_000}
P = {"use_cov": 1, "n_trees_used": 5}


def test_fp32_and_int32_peaks():
    r = bench.roofline({"lm": {"ms": 1.0, "launches": 1}}, WORK, P, 1, None, 152, PK)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.070e9 / 1e12)          # 80.5 TFLOP/s
    r = bench.roofline({"hypgen": {"ms": 1.0, "launches": 1}}, WORK, P, 1, None, 152, PK)
    assert r["unit"] == "Tops/s" and r["peak"] == pytest.approx(152 * 128 * 2.070e9 / 1e12)


def test_dominant_kernel_and_fraction():
    kernels = {"lm": {"ms": 12.0, "launches": 6}, "energy": {"ms": 2.0, "launches": 7},
               "raycast_score": {"ms": 1.5, "launches": 1}}
    r = bench.roofline(kernels, WORK, P, 64, None, 152, PK, batch=64)
    assert r["kernel"] == "lm" and r["bound"] == "alu"
    flops = 18 * 3000 + 18 * 120000 + 190 * 2000 + 34 * 1500
    assert r["avg_launch_ms"] == pytest.approx(2.0)
    assert r["achieved"] == pytest.approx(flops / 6 / 2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    k = bench.kernel_rooflines(kernels, WORK, P, 152, PK)
    assert k["energy"]["achieved"] == pytest.approx((20 * 1000 + 18 * 40000) / 2e-3 / 1e12)
    assert k["raycast_score"]["achieved"] == pytest.approx(45 * 10_000_000 / 1.5e-3 / 1e12)


def test_euclidean_modes_cost_nine_flops():
    e18 = bench.algorithmic_flops("energy", WORK, {"use_cov": 1})
    e9 = bench.algorithmic_flops("energy", WORK, {"use_cov": 0})
    assert e18 - e9 == 9 * WORK["energy_modes"]


def test_traffic_only_for_the_profiled_source():
    e = bench.PROFILED_TRAFFIC["lm"]
    path = os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), e["source"])
    with open(path, "rb") as f:
        same = hashlib.sha256(f.read()).hexdigest()[:16] == e["sha256_16"]
    t = bench.profiled_traffic("lm", 64)
    assert (t == pytest.approx(e["bytes_per_frame_launch"] * 64)) if same else t is None
    assert bench.profiled_traffic("energy", 64) is None


def test_end_to_end_roofline():
    r = bench.end_to_end_roofline(WORK, P, 64, 0.02, 152, PK)
    flops = (20 * 1000 + 18 * 40000) + (18 * 3000 + 18 * 120000 + 190 * 2000 + 34 * 1500) + 45 * 10_000_000
    assert r["flops_per_frame"] == pytest.approx(flops / 64)
    assert r["roofline_frames_per_s"] == pytest.approx(152 * 128 * 2 * 2.070e9 / (flops / 64))
    assert r["frac"] == pytest.approx((64 / 0.02) / r["roofline_frames_per_s"])
