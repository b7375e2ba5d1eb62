"""Hybrid cached replay on the GPU (Sec. 4.4) against the oracle's hybrid replay with the
same checkpoint interval k and thresholds (gamma, eps), through the C ABI.

Thresholds are chosen where the route decisions cannot flip between FP32 and FP64:
gamma = 0 never takes the scalar route; eps = +inf never inverts (every non-checkpoint
suffix recomputed: the exact gradient); eps = 1e-3 inverts only blocks whose |det| is far
from it (polarizers and diffuse bounces have det 0, retarders det 1).  The scalar route is
tested on the diffuse furnace, where every block throughput has DI = 0 exactly.  Every
schedule runs the hybrid: the megakernels trace a recomputed block again, the wavefront
re-shades it from the hits it keeps per vertex."""

import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg
from parity import GRAD_TOL, grad_rel, identical_path_pixels

pytestmark = pytest.mark.gpu

INF = float("inf")


@pytest.fixture(scope="module")
def env(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13265_gb300 import build, api
    build.build()
    dctx = api.Context(0)
    return api, dctx, oracle_mod


def _scenes():
    out = {"deep": sg.deep_stack_scene(num_sheets=85, width=12, height=8, spp=2, depth=128, tex_res=16, mesh=False),
           "mixed": sg.mixed_scene(width=16, spp=4, depth=6)}
    s, j = sg.rocks_scene(freq=4, num_rocks=3, tex_res=16, width=16, spp=4, depth=16)
    out["rocks"] = (s, j)
    return out


SCENES = _scenes()
CONFIGS = [(4, 0.0, INF), (8, 0.0, 1e-3), (16, 0.0, INF)]


def _adjoint_input(api, dctx, scene, job, O, seed):
    """Seeded dI restricted to pixels whose adjoint paths are identical on both sides."""
    gs = api.GpuScene(dctx, scene)
    frac, keep = identical_path_pixels(api, dctx, gs, job, O.OracleScene(scene), None)
    assert frac >= 0.85, frac   # 128-vertex paths part more often between FP32 and FP64
    return np.random.default_rng(seed).normal(size=(job.num_angles, job.num_pixels, 3, 4)) * keep[None, :, None, None]


def _gpu_grad(api, dctx, scene, job, dI, sched, k, gamma, eps):
    import torch
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    prev = dctx.get_launch()
    dctx.set_launch(sched, 128, 0)
    dctx.set_replay(k, gamma, eps)
    try:
        d_img = torch.as_tensor(dI.ravel(), dtype=torch.float32, device="cuda")
        g = api.render_adjoint(dctx, gs, batch, P, d_img)
        dctx.sync_status()
    finally:
        dctx.set_replay(1)
        dctx.set_launch(*prev)
    return {k_: v.double().cpu().numpy() for k_, v in g.items()}


def _compare(scene, got, ref, name):
    checked = 0
    for t, (off, w, h, ch) in enumerate(scene.tex_desc):
        if not scene.tex_differentiable[t]:
            continue
        o, g = ref["tex"][off:off + w * h * ch], got["tex"][off:off + w * h * ch]
        if np.linalg.norm(o) == 0:
            continue
        assert grad_rel(g, o) <= GRAD_TOL, (name, "tex", t, grad_rel(g, o))
        checked += 1
    for key in ("ior", "le", "sheet", "theta"):
        o = ref[key]
        if o.size == 0 or np.linalg.norm(o) == 0:
            continue
        assert grad_rel(got[key][:o.size], o) <= GRAD_TOL, (name, key, grad_rel(got[key][:o.size], o))
        checked += 1
    assert checked >= 2


# the sweep schedule runs the hybrid replay as the wavefront schedule
@pytest.mark.parametrize("sched", [0, 1, 2, 3], ids=["grid", "persistent", "wavefront", "sweep"])
@pytest.mark.parametrize("cfg", CONFIGS, ids=[f"k{c[0]}_eps{c[2]}" for c in CONFIGS])
@pytest.mark.parametrize("name", list(SCENES))
def test_hybrid_matches_oracle(env, name, cfg, sched):
    api, dctx, O = env
    scene, job = SCENES[name]
    job.pass_id = 1
    try:
        dI = _adjoint_input(api, dctx, scene, job, O, 7)
        got = _gpu_grad(api, dctx, scene, job, dI, sched, *cfg)
        ref, routes = O.OracleScene(scene).gradient_hybrid(job, scene.params(), dI, *cfg)
    finally:
        job.pass_id = 0
    assert routes["recompute"] + routes["inverse"] > 0
    _compare(scene, got, ref, name)


@pytest.mark.parametrize("sched", [0, 2], ids=["grid", "wavefront"])
def test_hybrid_exact_routes_equal_cached_replay(env, sched):
    """With eps = +inf the hybrid is exact: it matches the oracle's fully cached replay."""
    api, dctx, O = env
    scene, job = SCENES["deep"]
    job.pass_id = 1
    try:
        dI = _adjoint_input(api, dctx, scene, job, O, 3)
        got = _gpu_grad(api, dctx, scene, job, dI, sched, 8, 0.0, INF)
        ref = O.OracleScene(scene).gradient(job, scene.params(), dI, mode="replay")
    finally:
        job.pass_id = 0
    _compare(scene, got, ref, "deep")


@pytest.mark.parametrize("sched", [0, 2], ids=["grid", "wavefront"])
def test_hybrid_scalar_route_on_furnace(env, sched):
    """Every block of the diffuse furnace is an ideal depolarizer: the scalar PRB route is
    taken for every non-checkpoint vertex and is exact."""
    api, dctx, O = env
    scene, job = sg.furnace_scene(0.6, 1.5)
    job.max_depth = 30
    job.pass_id = 1
    dI = np.random.default_rng(4).normal(size=(job.num_angles, job.num_pixels, 3, 4))
    got = _gpu_grad(api, dctx, scene, job, dI, sched, 4, 0.5, INF)
    _, routes = O.OracleScene(scene).gradient_hybrid(job, scene.params(), dI, 4, 0.5, INF)
    ref = O.OracleScene(scene).gradient(job, scene.params(), dI, mode="tape")
    assert routes["scalar"] > 0 and routes["recompute"] == 0
    o, g = ref["tex"], got["tex"][:ref["tex"].size]
    assert grad_rel(g, o) <= GRAD_TOL


def test_hybrid_settings_and_errors(env):
    api, dctx, _ = env
    from paper_2607_13265_gb300 import _lib
    for bad in [(3, 0.0, 1.0), (0, 0.0, 1.0), (8, -1.0, 1.0), (8, 0.0, float("nan"))]:
        with pytest.raises(_lib.DpptError):
            dctx.set_replay(*bad)
    assert dctx.get_replay()[0] == 1
    scene, job = sg.mixed_scene(width=8, spp=2, depth=6)
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    import torch
    prev = dctx.get_launch()
    dctx.set_replay(1, method="pprb", sigma=0.01)
    try:
        # P-PRB has no wavefront form, and the sweep schedule replays in waves
        for sched in (2, 3):
            dctx.set_launch(sched, 128, 0)
            with pytest.raises(_lib.DpptError, match="UNSUPPORTED"):
                api.render_adjoint(dctx, gs, batch, P, torch.zeros(batch.image_floats, device="cuda"))
    finally:
        dctx.set_replay(1)
        dctx.set_launch(*prev)


def test_hybrid_footprint_is_smaller(env):
    api, dctx, _ = env
    prev = dctx.get_launch()
    dctx.set_launch(0, 128, 0)
    try:
        full = dctx.adjoint_footprint(128)
        dctx.set_replay(16, 0.0, INF)
        hyb = dctx.adjoint_footprint(128)
    finally:
        dctx.set_replay(1)
        dctx.set_launch(*prev)
    assert full["local_bytes_per_thread"] >= 128 * 124
    assert hyb["local_bytes_per_thread"] < 0.5 * full["local_bytes_per_thread"]


def test_wavefront_hybrid_workspace_and_primal(env):
    """The wavefront with k = 16 keeps each vertex's hit and the checkpoint data instead of
    the 144-byte cached vertex: at depth 128 its workspace is at most half the cached
    replay's.  Its primal waves fold over blocks; the image equals the cached primal's to
    FP32 rounding."""
    import torch
    from parity import image_rel_err, flat
    api, dctx, _ = env
    scene, job = SCENES["deep"]
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    P = api.device_params(scene, batch)
    prev = dctx.get_launch()
    dctx.set_launch(2, 128, 0)
    try:
        full = dctx.query_workspace(batch)
        img_full = api.image_views(batch, api.render_primal(dctx, gs, batch, P))[0].double().cpu().numpy()
        dctx.set_replay(16, 0.0, INF)
        hyb = dctx.query_workspace(batch)
        img_hyb = api.image_views(batch, api.render_primal(dctx, gs, batch, P))[0].double().cpu().numpy()
        dctx.sync_status()
    finally:
        dctx.set_replay(1)
        dctx.set_launch(*prev)
    assert hyb <= 0.5 * full, (hyb, full)
    assert float(image_rel_err(flat(img_hyb), flat(img_full)).max()) <= 1e-4
