"""The library's tuning and accounting entry points through the C ABI: the autotuner,
the instrumented work count, the workspace query, the per-stage launch statistics and the
scene summary, checked against the oracle's counts on the same seeded paths and against
the scene itself."""
import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg
from parity import gpu_image, grad_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13265_gb300 import build, api
    build.build()
    return api, api.Context(0), oracle_mod


def test_scene_info_matches_scene(env):
    api, dctx, _ = env
    scene, _ = sg.cornell_box()
    gs = api.GpuScene(dctx, scene)
    info = gs.info()
    assert info["triangles"] == scene.num_triangles
    assert info["spheres"] == 2
    assert info["bvh_nodes"] >= 1 and 1 <= info["bvh_depth"] < 64
    assert info["device_bytes"] > 0


def test_work_count_matches_oracle(env):
    """Rays, shadow rays and surface vertices of the jobs' paths: the instrumented GPU walk
    and the FP64 oracle walk the same paths, so the counts agree up to the few paths whose
    FP32 and FP64 walks part."""
    api, dctx, O = env
    scene, job = sg.icosphere_scene(freq=8, tex_res=16, width=32, spp=8, depth=8)
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    w = api.count_work(dctx, gs, batch, P)
    O.stats(reset=True)
    O.OracleScene(scene).render(job, scene.params())
    o = O.stats(reset=True)
    assert w["paths"] == job.num_paths == int(o["paths"])
    for k in ("rays", "shadow_rays", "vertices"):
        assert abs(w[k] - o[k]) <= 0.01 * o[k], (k, w[k], o[k])
    assert w["rays"] >= w["paths"] and w["vertices"] <= w["rays"]
    assert w["nodes"] > 0 and w["tri_tests"] > 0


def test_workspace_grows_with_depth_in_the_wavefront(env):
    api, dctx, _ = env
    _, job = sg.cornell_box()
    prev = dctx.get_launch()
    try:
        dctx.set_launch(2, 128, 0)
        sizes = []
        for d in (2, 8, 32):
            job.max_depth = d
            sizes.append(dctx.query_workspace(api.pack_jobs([job])))
        dctx.set_launch(0, 128, 0)
        grid = dctx.query_workspace(api.pack_jobs([job]))
        dctx.set_launch(3, 128, 0)      # the sweep's adjoint keeps the wavefront's waves
        sweep = dctx.query_workspace(api.pack_jobs([job]))
    finally:
        dctx.set_launch(*prev)
    assert sizes[0] < sizes[1] < sizes[2] == sweep
    # the cache grows by 144 bytes per vertex and path (64x64 pixels x 16 spp)
    assert sizes[2] - sizes[1] >= 24 * 144 * job.num_paths
    assert grid < sizes[0]


def test_stage_statistics_count_launches(env):
    api, dctx, _ = env
    scene, job = sg.cornell_box()
    gs = api.GpuScene(dctx, scene)
    prev = dctx.get_launch()
    try:
        dctx.set_launch(2, 128, 0)
        dctx.stage_stats(timing=True, reset=True)
        gpu_image(api, dctx, gs, [job])
        st = dctx.stage_stats(timing=False, reset=True)
        dctx.set_launch(0, 128, 0)
        gpu_image(api, dctx, gs, [job])
        st_grid = dctx.stage_stats(timing=False, reset=True)
    finally:
        dctx.set_launch(*prev)
    # one wave, depth 4: four extend + shade, shadow and cache launches, one pixel sum
    assert st["wf_extend"][0] == job.max_depth and st["wf_shadow"][0] == job.max_depth
    assert st["wf_cache"][0] == job.max_depth and st["wf_pixels"][0] == 1
    assert st["wf_extend"][1] > 0.0
    assert st["primal"][0] == 0 and st_grid["primal"][0] == 1
    assert st_grid["wf_extend"][0] == 0


def test_stage_statistics_of_the_sweep_schedule(env):
    """The sweep schedule's adjoint: one forward-sweep megakernel per wave, then max_depth
    replay iterations (every path starts its replay at the first), one pixel sum; none of
    the forward sweep's stage kernels.  Its primal is the grid schedule's megakernel."""
    import torch
    api, dctx, _ = env
    scene, job = sg.cornell_box()
    gs = api.GpuScene(dctx, scene)
    prev = dctx.get_launch()
    try:
        dctx.set_launch(3, 128, 0)
        dctx.stage_stats(timing=False, reset=True)
        (img,), batch, P = gpu_image(api, dctx, gs, [job])
        st_p = dctx.stage_stats(timing=False, reset=True)
        dI = torch.ones(img.size, dtype=torch.float32, device="cuda")
        api.render_adjoint(dctx, gs, batch, P, dI)
        dctx.sync_status()
        st = dctx.stage_stats(timing=False, reset=True)
    finally:
        dctx.set_launch(*prev)
    assert st_p["primal"][0] == 1 and st_p["wf_sweep"][0] == 0
    assert st["wf_sweep"][0] == 1 and st["wf_pixels"][0] == 1
    assert st["wf_extend"][0] == st["wf_shadow"][0] == st["wf_cache"][0] == 0
    assert st["primal"][0] == st["adjoint"][0] == 0
    n = st["wf_replay"][0]
    assert n >= job.max_depth and n % job.max_depth == 0


def test_adjoint_footprint_follows_the_schedule(env):
    """Under the sweep schedule the footprint is the forward-sweep megakernel's: its
    thread-local arrays hold E_v and W_v (31 floats) per vertex of the cache depth, and at
    most 256 threads a block (a 512-thread shape runs its sweep at 256)."""
    api, dctx, _ = env
    prev = dctx.get_launch()
    try:
        dctx.set_launch(0, 256, 0, 3, 512, 0)
        sw = dctx.adjoint_footprint(8)
        dctx.set_launch(0, 256, 0, 0, 256, 0)
        mk = dctx.adjoint_footprint(8)
    finally:
        dctx.set_launch(*prev)
    assert sw["local_bytes_per_thread"] >= 8 * 31 * 4 and mk["local_bytes_per_thread"] >= 8 * 31 * 4
    assert sw["registers"] <= 128 and sw["threads_per_sm"] % 256 == 0 and 256 <= sw["threads_per_sm"] <= 2048
    assert sw["threads_per_sm"] >= mk["threads_per_sm"]      # the primal's launch bounds, not the adjoint's
    assert sw["sms"] == mk["sms"] > 0


def test_autotune_picks_valid_shapes_with_equal_results(env):
    import torch
    api, dctx, _ = env
    scene, job = sg.mixed_scene(width=24, spp=4, depth=6)
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    prev = dctx.get_launch()
    try:
        dctx.set_launch(0, 128, 0)
        (ref,), _, _ = gpu_image(api, dctx, gs, [job])
        dI = torch.as_tensor(np.random.default_rng(3).normal(size=ref.size), dtype=torch.float32, device="cuda")
        g_ref = {k: v.double().cpu().numpy() for k, v in api.render_adjoint(dctx, gs, batch, P, dI).items()}
        t = api.autotune(dctx, gs, batch, P, reps=1)
        assert t["primal"][0] in ("grid", "persistent", "wavefront") and t["primal"][1] in (64, 128, 256)
        assert t["adjoint"][0] in ("grid", "persistent", "wavefront", "sweep") and t["adjoint"][1] in (64, 128, 256)
        assert all(np.isinf(t["times_ms"][f"sweep/{b}"]["primal_ms"]) for b in (64, 128, 256))
        assert all(np.isfinite(t["times_ms"][f"sweep/{b}"]["adjoint_ms"]) for b in (64, 128, 256))
        assert t["adjoint_scatter"] in ("warp", "lane")
        timed = [v for v in t["times_ms"].values() if v["primal_ms"] > 0]
        assert len(timed) >= 3
        lc = dctx.get_launch()
        assert api.SCHEDULE_NAMES[lc[0]] == t["primal"][0] and lc[1] == t["primal"][1]
        (got,), _, _ = gpu_image(api, dctx, gs, [job])
        g = {k: v.double().cpu().numpy() for k, v in api.render_adjoint(dctx, gs, batch, P, dI).items()}
        dctx.sync_status()
    finally:
        dctx.set_launch(*prev)
    assert np.allclose(ref, got, rtol=1e-5, atol=1e-6 * np.abs(ref).max())
    for k in ("tex", "le"):
        assert grad_rel(g[k], g_ref[k]) <= 1e-4, (k, grad_rel(g[k], g_ref[k]))
