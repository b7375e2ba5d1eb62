"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs.  Images: per-pixel relative error (tests/parity.py) at the 99.9th
percentile <= 1e-4, paths compared one by one through their signatures.  Gradients
(cached suffix replay on the GPU vs the oracle): relative L2 error <= 1e-3 per parameter
group, and per element for the scalar groups."""
import math

import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg
from parity import IMG_TOL_P999, GRAD_TOL, image_rel_err, gpu_image, flat, grad_rel, identical_path_pixels, \
    scalar_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13265_gb300 import build, api
    build.build()
    dctx = api.Context(0)
    return api, dctx, oracle_mod


def small_scenes():
    out = {}
    s, j = sg.cornell_box()
    j.width = j.height = 32
    out["cornell"] = (s, j)
    out["mixed"] = sg.mixed_scene(width=24, spp=4, depth=6)
    s, j = sg.icosphere_scene(freq=8, tex_res=16, width=32, spp=8, depth=8)
    out["icosphere"] = (s, j)
    s, j = sg.rocks_scene(freq=4, num_rocks=3, tex_res=16, width=20, spp=4, depth=16)
    out["rocks"] = (s, j)
    # 85 stacked polarizers in a closed room with a curved rough conductor: paths of up to 128
    # vertices (largest cache bucket)
    out["deep"] = sg.deep_stack_scene(num_sheets=85, width=12, height=8, spp=2, depth=128, tex_res=16)
    # normal maps on a rough dielectric, a diffuse and a rough conductor surface
    out["nmap"] = sg.normal_map_scene(width=20, spp=4, depth=4, tex_res=16)
    # thirteen polarized lights: 156 scalar gradients, more than the 32 shared-memory copies
    # per scalar fit in 16 KB, so the kernels keep one copy of each
    s, j = sg.cornell_box()
    for k in range(12):
        a = 2.0 * np.pi * k / 12
        s.add_light((0.7 * np.cos(a) - 0.06, 0.998, 0.7 * np.sin(a) - 0.06), (0.12, 0, 0), (0, 0, 0.12),
                    [[4.0, 1.0, 0.5, 0.2]] * 3)
    j.width = j.height = 24
    out["lights13"] = (s, j)
    # the closed-form scenes of the oracle's pins: NEE + MIS from two lights, the same quads
    # as emitting surfaces, one interface seen from the medium's side, a glass slab, and a
    # roughness-0.01 conductor under a small polarized light
    out["polylight"] = sg.polygon_light_scene(spp=256)
    out["emitters"] = sg.polygon_light_scene(surface_emission=True, spp=256)
    out["glass_in"] = sg.glass_interface_scene(camera_inside=True, spp=64)
    out["slab"] = sg.glass_interface_scene(slab=0.2, spp=64)
    out["specular"] = sg.specular_limit_scene("conductor", 50.0, spp=256, light_size=0.4)
    return out


# fraction of paths that must be identical between FP32 and FP64.  Position errors grow
# along a path (a bounce at incidence cosine c scales the error parallel to the wall by
# ~1/c), so long paths in a closed room part more often: about 6% of the 128-vertex paths
# of the deep scene (22% in the same room without the stack, more where a path meets the
# curved conductor) versus < 1% at depth 16.
MIN_IDENTICAL = {"deep": 0.85}


SCENES = small_scenes()


# the sweep schedule renders the primal as the grid schedule; its adjoint traces each wave in one
# forward-sweep megakernel and replays it with the wavefront's kernels
SCHEDULES = {"grid": (0, 128), "persistent": (1, 256), "wavefront": (2, 128), "sweep": (3, 128)}


@pytest.fixture(params=list(SCHEDULES))
def sched(request, env):
    _, dctx, _ = env
    prev = dctx.get_launch()
    dctx.set_launch(*SCHEDULES[request.param], 0)
    yield request.param
    dctx.set_launch(*prev)


@pytest.mark.parametrize("name", list(SCENES))
def test_primal_matches_oracle(env, sched, name):
    api, dctx, O = env
    scene, job = SCENES[name]
    gs = api.GpuScene(dctx, scene)
    (g,), sig_g, _, _ = gpu_image(api, dctx, gs, [job], with_sig=True)
    o, _, sig_o = O.OracleScene(scene).render(job, scene.params(), paths=True)
    g = flat(g)
    assert np.abs(o).max() > 0
    same_path = sig_g == sig_o
    assert same_path.mean() >= MIN_IDENTICAL.get(name, 0.99), f"only {same_path.mean():.4f} of the paths are identical"
    err = image_rel_err(g, o)
    pix_ok = same_path.reshape(-1, job.spp).all(1)
    p999 = float(np.quantile(err[:, pix_ok], 0.999))
    assert p999 <= IMG_TOL_P999, f"p99.9 relative error {p999:.3g}"
    assert float(err[:, pix_ok].max()) <= 10 * IMG_TOL_P999


@pytest.mark.parametrize("name", list(SCENES))
def test_adjoint_matches_oracle(env, sched, name):
    import torch
    api, dctx, O = env
    scene, job = SCENES[name]
    job.pass_id = 1
    try:
        gs = api.GpuScene(dctx, scene)
        batch = api.pack_jobs([job])
        P = api.device_params(scene, batch)
        frac, keep = identical_path_pixels(api, dctx, gs, job, O.OracleScene(scene), None)
        assert frac >= MIN_IDENTICAL.get(name, 0.99), frac
        rng = np.random.default_rng(7)
        dI = rng.normal(size=(job.num_angles, job.num_pixels, 3, 4)) * keep[None, :, None, None]
        d_img = torch.as_tensor(dI.ravel(), dtype=torch.float32, device="cuda")
        grads = api.render_adjoint(dctx, gs, batch, P, d_img)
        dctx.sync_status()
        ref = O.OracleScene(scene).gradient(job, scene.params(), dI, mode="replay")
    finally:
        job.pass_id = 0
    got = {k: v.double().cpu().numpy() for k, v in grads.items()}
    checked = 0
    for t, (off, w, h, ch) in enumerate(scene.tex_desc):
        if not scene.tex_differentiable[t]:
            continue
        o, g = ref["tex"][off:off + w * h * ch], got["tex"][off:off + w * h * ch]
        if np.linalg.norm(o) == 0:
            continue
        assert grad_rel(g, o) <= GRAD_TOL, (name, "tex", t, grad_rel(g, o))
        checked += 1
    for k in ("ior", "le", "sheet", "theta"):
        o = ref[k]
        if o.size == 0 or np.linalg.norm(o) == 0:
            continue
        g = got[k][:o.size]
        assert grad_rel(g, o) <= GRAD_TOL, (name, k, g, o)
        assert float(scalar_rel(g, o).max()) <= GRAD_TOL, (name, k, scalar_rel(g, o), g, o)
        checked += 1
    # the emitting-surface scene has no quad light: its floor albedo is the one group
    assert checked >= (1 if name == "emitters" else 2)


def test_malus_on_gpu(env):
    import torch
    api, dctx, O = env
    for alpha, theta in [(0.3, 1.1), (1.0, -0.4)]:
        scene, job = sg.malus_scene(alpha, le=2.0)
        job.thetas = [theta]
        gs = api.GpuScene(dctx, scene)
        (img,), batch, P = gpu_image(api, dctx, gs, [job])
        assert np.allclose(img[..., 0, 0], math.cos(theta - alpha) ** 2, rtol=1e-5)
        job.pass_id = 1
        batch = api.pack_jobs([job])
        d = torch.zeros(batch.image_floats, device="cuda")
        d.view(-1, 3, 4)[:, 0, 0] = 1.0
        g = api.render_adjoint(dctx, gs, batch, P, d)
        expect = -math.sin(2 * (theta - alpha)) * job.num_pixels
        assert g["theta"][0].item() == pytest.approx(expect, rel=1e-4, abs=1e-5)
        assert g["sheet"][0].item() == pytest.approx(-expect, rel=1e-4, abs=1e-5)


def test_furnace_on_gpu(env):
    api, dctx, _ = env
    scene, job = sg.furnace_scene(0.6, 1.5)
    gs = api.GpuScene(dctx, scene)
    for depth in (1, 3, 7, 100, 128):
        job.max_depth = depth
        (img,), _, _ = gpu_image(api, dctx, gs, [job])
        assert np.allclose(img[..., 0], 1.5 * sum(0.6**k for k in range(depth)), rtol=2e-6)
        assert np.all(img[..., 1:] == 0.0)


def test_diffuse_depolarizes_on_gpu(env):
    api, dctx, _ = env
    scene, job = sg.cornell_box()
    scene.spheres, scene.sph_mat = scene.spheres[:1], scene.sph_mat[:1]
    job.filter, job.thetas = sg.FILTER_NONE, []
    gs = api.GpuScene(dctx, scene)
    (img,), _, _ = gpu_image(api, dctx, gs, [job])
    assert img[..., 0].max() > 0 and np.all(img[..., 1:] == 0.0)


def test_batched_angles_equal_separate_jobs(env):
    """One job with a batch of polarizer angles equals one job per angle (the camera
    filter does not change the paths, so the fold is exact)."""
    import copy
    import torch
    api, dctx, _ = env
    scene, job = sg.cornell_box()
    job.width = job.height = 24
    thetas = [0.1, 0.9, 2.0, 3.0]
    job.thetas = thetas
    gs = api.GpuScene(dctx, scene)
    (batched,), bb, Pb = gpu_image(api, dctx, gs, [job])
    singles = []
    for t in thetas:
        j = copy.copy(job)
        j.thetas = [t]
        singles.append(j)
    views, sb, Ps = gpu_image(api, dctx, gs, singles)
    for a in range(len(thetas)):
        assert np.allclose(batched[a], views[a][0], rtol=1e-6, atol=1e-7)
    # adjoint: theta gradients of the batched job equal those of the single jobs
    for j in [job] + singles:
        j.pass_id = 1
    bb, sb = api.pack_jobs([job]), api.pack_jobs(singles)
    rng = np.random.default_rng(3)
    d = torch.as_tensor(rng.normal(size=bb.image_floats), dtype=torch.float32, device="cuda")
    gb = api.render_adjoint(dctx, gs, bb, Pb, d)
    gsum = api.render_adjoint(dctx, gs, sb, Ps, d)
    assert np.allclose(gb["theta"].cpu().numpy(), gsum["theta"].cpu().numpy(), rtol=1e-4, atol=1e-5)
    tex_b, tex_s = gb["tex"].cpu().numpy(), gsum["tex"].cpu().numpy()
    assert np.linalg.norm(tex_b - tex_s) <= 1e-4 * np.linalg.norm(tex_s)


@pytest.mark.parametrize("schedule,block", [(0, 64), (0, 256), (1, 128), (1, 256), (2, 64), (2, 256), (3, 256)])
def test_schedules_agree(env, schedule, block):
    api, dctx, _ = env
    scene, job = SCENES["mixed"]
    gs = api.GpuScene(dctx, scene)
    prev = dctx.get_launch()
    try:
        dctx.set_launch(0, 128, 0)
        (ref,), _, _ = gpu_image(api, dctx, gs, [job])
        dctx.set_launch(schedule, block, 0)
        (got,), _, _ = gpu_image(api, dctx, gs, [job])
    finally:
        dctx.set_launch(*prev)
    if schedule == 2:   # another schedule of the same arithmetic: equal up to summation order
        assert np.allclose(ref, got, rtol=1e-5, atol=1e-6 * np.abs(ref).max())
    else:            # same kernel, deterministic per-pixel sums: bitwise equal
        assert np.array_equal(ref, got)


@pytest.mark.parametrize("depth", [1, 2])
def test_shallow_paths(env, sched, depth):
    """Depth 1 (emitter hits only, no light samples) and depth 2: the edge cases of the
    wavefront's iteration count and of the replay's first and last vertex."""
    import torch
    api, dctx, O = env
    scene, job = sg.cornell_box()
    job.width = job.height = 24
    job.max_depth = depth
    job.pass_id = 1
    try:
        gs = api.GpuScene(dctx, scene)
        batch = api.pack_jobs([job])
        P = api.device_params(scene, batch)
        frac, keep = identical_path_pixels(api, dctx, gs, job, O.OracleScene(scene), None)
        assert frac >= 0.99, frac
        (g_img,), _, _ = gpu_image(api, dctx, gs, [job])
        o_img = O.OracleScene(scene).render(job, scene.params())
        dI = np.random.default_rng(11).normal(size=(job.num_angles, job.num_pixels, 3, 4)) * keep[None, :, None, None]
        grads = api.render_adjoint(dctx, gs, batch, P, torch.as_tensor(dI.ravel(), dtype=torch.float32, device="cuda"))
        dctx.sync_status()
        ref = O.OracleScene(scene).gradient(job, scene.params(), dI, mode="replay")
    finally:
        job.pass_id = 0
    err = image_rel_err(flat(g_img), o_img)[:, keep]
    assert float(np.quantile(err, 0.999)) <= IMG_TOL_P999
    got = {k: v.double().cpu().numpy() for k, v in grads.items()}
    keys = ("le", "theta") if depth == 1 else ("tex", "le", "theta")
    for k in keys:
        o = ref[k]
        assert np.linalg.norm(o) > 0, k
        assert grad_rel(got[k][:o.size], o) <= GRAD_TOL, (k, grad_rel(got[k][:o.size], o))
    if depth == 1:      # nothing scatters at depth 1: no texture or index-of-refraction gradient
        assert np.all(got["tex"] == 0.0) and np.all(ref["tex"] == 0.0)


def test_wavefront_waves_match_megakernel(env):
    """A job of 7.84 M paths runs as two wavefront waves (at most 4,194,304 paths each, whole
    pixels), by the stage kernels and by the sweep schedule's forward-sweep megakernel: image
    and gradients equal the grid megakernel's, which has no waves, up to
    summation order.  A gradient element sums millions of FP32 atomic additions in an order
    that differs between the schedules (about sqrt(N) * 6e-8 ~ 2e-4 relative at N = 8e6);
    a lost or repeated wave would be an O(1) error."""
    import torch
    api, dctx, _ = env
    scene, job = sg.cornell_box()
    job.width = job.height = 700
    job.spp, job.max_depth = 16, 4
    assert job.num_paths > 4194304
    gs = api.GpuScene(dctx, scene)
    prev = dctx.get_launch()
    out = []
    try:
        for sched in (0, 2, 3):
            dctx.set_launch(sched, 128, 0, sched, 128, 0)
            (img,), batch, P = gpu_image(api, dctx, gs, [job])
            dI = torch.as_tensor(np.random.default_rng(5).normal(size=img.size), dtype=torch.float32, device="cuda")
            g = api.render_adjoint(dctx, gs, batch, P, dI)
            dctx.sync_status()
            out.append((img, {k: v.double().cpu().numpy() for k, v in g.items()}))
    finally:
        dctx.set_launch(*prev)
    (ri, rg), *waved = out
    assert np.abs(ri).max() > 0
    for wi, wg in waved:
        assert np.allclose(ri, wi, rtol=1e-5, atol=1e-6 * np.abs(ri).max())
        for k in ("tex", "ior", "le", "theta"):
            assert np.linalg.norm(rg[k]) > 0, k
            assert grad_rel(wg[k], rg[k]) <= GRAD_TOL, (k, grad_rel(wg[k], rg[k]))


@pytest.mark.parametrize("w,h,spp", [(37, 23, 3), (19, 5, 64), (1, 1, 1), (7, 9, 33)])
def test_ragged_sizes(env, sched, oracle_mod, w, h, spp):
    api, dctx, O = env
    scene, job = sg.mixed_scene(width=8, spp=1, depth=5)
    job.width, job.height, job.spp = w, h, spp
    gs = api.GpuScene(dctx, scene)
    (g,), sig, _, _ = gpu_image(api, dctx, gs, [job], with_sig=True)
    o, _, sig_o = O.OracleScene(scene).render(job, scene.params(), paths=True)
    err = image_rel_err(flat(g), o)
    pix_ok = (sig == sig_o).reshape(-1, spp).all(1)
    assert pix_ok.mean() >= 0.95
    assert float(err[:, pix_ok].max()) <= 10 * IMG_TOL_P999


def test_empty_and_invalid(env):
    import torch
    api, dctx, _ = env
    from paper_2607_13265_gb300 import _lib
    scene, job = sg.cornell_box()
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([])
    P = api.device_params(scene, api.pack_jobs([job]))
    api.render_primal(dctx, gs, batch, P, image=torch.zeros(1, device="cuda"))   # no jobs: no-op
    for field, value in [("camera", 5), ("max_depth", 0), ("max_depth", 129), ("spp", 0), ("filter", 9)]:
        bad = api.pack_jobs([job])
        setattr(bad.c_jobs[0], field, value)
        with pytest.raises(_lib.DpptError):
            api.render_primal(dctx, gs, bad, P)
    with pytest.raises(_lib.DpptError):
        dctx.set_launch(0, 100, 0)
    dctx.sync_status()


def test_full_size_workload_sampled_pixels(env):
    """The 256x256, 64 spp, depth 8 icosphere workload in the launch configuration the
    benchmark times; 48 sampled pixels recomputed by the oracle one by one."""
    api, dctx, O = env
    scene, job = sg.icosphere_scene()
    gs = api.GpuScene(dctx, scene)
    (g,), sig, _, _ = gpu_image(api, dctx, gs, [job], with_sig=True)
    rng = np.random.default_rng(11)
    pix = np.sort(rng.choice(job.num_pixels, 48, replace=False))
    o, _, sig_o = O.OracleScene(scene).render(job, scene.params(), pixels=pix, paths=True)
    gp = flat(g)[:, pix]
    sig_g = sig.reshape(-1, job.spp)[pix].ravel()
    same = (sig_g == sig_o).reshape(-1, job.spp).all(1)
    assert same.mean() >= 0.9
    err = image_rel_err(gp, o)
    assert float(err[:, same].max()) <= 10 * IMG_TOL_P999


@pytest.mark.parametrize("sched", [0, 2], ids=["grid", "wavefront"])
def test_texel_scatter_modes_agree(env, sched):
    """Texel gradients combined per warp group or issued one atomic per lane: the same sums
    in another order."""
    import torch
    api, dctx, _ = env
    scene, job = SCENES["icosphere"]
    gs = api.GpuScene(dctx, scene)
    adj = api.pack_jobs(api.adjoint_jobs([job]))
    P = api.device_params(scene, adj)
    d = torch.as_tensor(np.random.default_rng(3).normal(size=adj.image_floats), dtype=torch.float32, device="cuda")
    prev = dctx.get_launch()
    out = []
    try:
        for scatter in (0, 1):
            dctx.set_launch(sched, 128, 0, sched, 128, 0, scatter)
            out.append(api.render_adjoint(dctx, gs, adj, P, d)["tex"].double().cpu().numpy())
    finally:
        dctx.set_launch(*prev)
    assert np.linalg.norm(out[0]) > 0
    assert np.linalg.norm(out[0] - out[1]) <= 1e-5 * np.linalg.norm(out[0])
