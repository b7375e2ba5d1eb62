"""The benchmark's accounting, on CPU: the algorithmic flops each stage is charged with, and
the roofline of the stage with the most GPU time, including the DRAM traffic per launch
that ncu measured for the views workload's dominant kernels."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

WORK = {"paths": 1000, "vertices": 4000, "rays": 5000, "shadow_rays": 3000, "nodes": 90000, "shadow_nodes": 30000,
        "tri_tests": 20000, "shadow_tri_tests": 100, "sph_tests": 10000, "shadow_sph_tests": 6000}
PEAKS = {"hbm_gbs": 6775.6, "sm_max_mhz": 2070.0, "_source": "measured"}
PROPS = SimpleNamespace(multi_processor_count=152)


def traversal_flops(w, shadow):
    p = "shadow_" if shadow else ""
    return bench.F_NODE * w[p + "nodes"] + bench.F_TRI * w[p + "tri_tests"] + bench.F_SPH * w[p + "sph_tests"]


def test_stage_flops_charge_the_sweep_as_the_primal_megakernel():
    f2 = bench.stage_flops(WORK, 2)
    f1 = bench.stage_flops(WORK, 1)
    closest, shadow = traversal_flops(WORK, False), traversal_flops(WORK, True)
    assert f2["wf_sweep"] == pytest.approx(closest + shadow + WORK["vertices"] * bench.F_VERTEX_PRIMAL)
    assert f2["wf_sweep"] == pytest.approx(f1["primal"])
    assert f2["wf_replay"] == pytest.approx(WORK["vertices"] * (bench.F_REPLAY + bench.F_SHADE))
    assert "wf_sweep" not in f1 and "primal" not in f2


def test_workload_flops_of_the_sweep_schedule():
    """Grid primal and sweep adjoint: the primal's flops come from the primal work, the
    sweep's and the replay's from the adjoint work, and K steps count K times."""
    pwork = dict(WORK, vertices=3900)
    flops, cache_bytes = bench.workload_flops(WORK, pwork, (0, 256, 0, 3, 256, 0, 0), 5)
    assert flops["primal"] == pytest.approx(5 * bench.stage_flops(pwork, 1)["primal"])
    assert flops["wf_sweep"] == pytest.approx(5 * bench.stage_flops(WORK, 2)["wf_sweep"])
    assert "wf_shade" not in flops
    assert cache_bytes == pytest.approx(5 * bench.cache_pass_bytes(WORK, 2))


def test_roofline_of_the_dominant_stage():
    flops, cache_bytes = bench.workload_flops(WORK, WORK, (0, 256, 0, 3, 256, 0, 0), 5)
    stages = {"primal": (5, 90.0), "wf_sweep": (20, 100.0), "wf_replay": (480, 50.0), "wf_cache": (0, 0.0)}
    r = bench.roofline_of(stages, flops, cache_bytes, PROPS, PEAKS, {"sm_mhz": 2070.0}, bench.WORKLOAD, WORK)
    assert r["kernel"] == "wf_sweep" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    launch_s = 100.0 / 20 / 1e3
    assert r["achieved"] == pytest.approx(flops["wf_sweep"] / 20 / launch_s / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2070.0e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    traffic = bench.DRAM_BYTES_PER_LAUNCH[(bench.WORKLOAD, "wf_sweep")]
    assert r["traffic"] == traffic
    assert r["hbm"]["achieved_gbs"] == pytest.approx(traffic / launch_s / 1e9)
    assert r["hbm"]["frac"] == pytest.approx(r["hbm"]["achieved_gbs"] / PEAKS["hbm_gbs"])


def test_roofline_of_a_cache_pass_is_bound_by_hbm_and_unknown_traffic_is_null():
    flops, cache_bytes = bench.workload_flops(WORK, WORK, (2, 128, 0, 2, 64, 0, 1), 3)
    stages = {"wf_extend": (24, 10.0), "wf_cache": (24, 12.0), "wf_replay": (45, 6.0)}
    r = bench.roofline_of(stages, flops, cache_bytes, PROPS, PEAKS, {}, bench.ICO_WORKLOAD, WORK)
    assert r["kernel"] == "wf_cache" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(cache_bytes / 24 / (12.0 / 24 / 1e3) / 1e9)
    assert r["peak"] == PEAKS["hbm_gbs"] and r["traffic"] is None
