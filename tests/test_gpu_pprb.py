"""Basic polarized PRB on the GPU (Sec. 4.1-4.2; the baseline): against the oracle's P-PRB
(same noise stream, noise in both passes) where every factor is invertible, and the
failure reproduced on a polarizer stack where the cached suffix replay stays exact."""
import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg
from parity import GRAD_TOL, grad_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13265_gb300 import build, api
    build.build()
    return api, api.Context(0), oracle_mod


def _gpu_grad(api, dctx, scene, job, dI, method, sigma=0.0, sched=0):
    import torch
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    prev = dctx.get_launch()
    dctx.set_launch(sched, 128, 0)
    dctx.set_replay(method=method, sigma=sigma)
    try:
        g = api.render_adjoint(dctx, gs, batch, P, torch.as_tensor(dI.ravel(), dtype=torch.float32, device="cuda"))
        dctx.sync_status()
    finally:
        dctx.set_replay()
        dctx.set_launch(*prev)
    return {k: v.double().cpu().numpy() for k, v in g.items()}


@pytest.mark.parametrize("sched", [0, 1], ids=["grid", "persistent"])
def test_pprb_matches_oracle_on_invertible_factors(env, sched):
    api, dctx, O = env
    cases = [(sg.retarder_pair_scene(), "sheet"), (sg.furnace_scene(0.5, 1.0), "tex")]
    for (scene, job), key in cases:
        job.pass_id = 1
        if key == "tex":
            job.max_depth = 4
        dI = np.random.default_rng(2).normal(size=(job.num_angles, job.num_pixels, 3, 4))
        got = _gpu_grad(api, dctx, scene, job, dI, "pprb", 1e-3, sched)[key]
        ref = O.OracleScene(scene).gradient(job, scene.params(), dI, mode="pprb", sigma=1e-3)[key]
        assert np.linalg.norm(ref) > 0
        assert grad_rel(got[:ref.size], ref) <= GRAD_TOL, (key, grad_rel(got[:ref.size], ref))


def test_pprb_fails_on_polarizer_stack_where_cached_replay_is_exact(env):
    api, dctx, O = env
    scene, job = sg.polarizer_stack_scene([0.0, 0.4, 0.9, 1.3, 1.9])
    job.pass_id = 1
    dI = np.random.default_rng(1).normal(size=(job.num_angles, job.num_pixels, 3, 4))
    exact = O.OracleScene(scene).gradient(job, scene.params(), dI, mode="tape")["sheet"]
    cached = _gpu_grad(api, dctx, scene, job, dI, "cached")["sheet"][:exact.size]
    assert grad_rel(cached, exact) <= GRAD_TOL
    for sigma in (1e-1, 1e-2, 1e-3, 1e-4):
        g = _gpu_grad(api, dctx, scene, job, dI, "pprb", sigma)["sheet"][:exact.size]
        assert grad_rel(g, exact) > 0.05, (sigma, grad_rel(g, exact))


def test_pprb_memory_is_independent_of_depth(env):
    api, dctx, _ = env
    prev = dctx.get_launch()
    dctx.set_launch(0, 128, 0)
    try:
        cached = dctx.adjoint_footprint(64)["local_bytes_per_thread"]
        dctx.set_replay(method="pprb", sigma=1e-3)
        p8 = dctx.adjoint_footprint(8)["local_bytes_per_thread"]
        p64 = dctx.adjoint_footprint(64)["local_bytes_per_thread"]
    finally:
        dctx.set_replay()
        dctx.set_launch(*prev)
    assert p8 == p64 < 0.25 * cached
