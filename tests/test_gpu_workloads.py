"""GPU parity on the shapes of the batched and large workloads.

* Views x angles: the Cornell scene from three cameras with uneven image sizes, four
  polarizer angles per view and one unfiltered job, each job at its own output offset,
  rendered by ONE render_primal and differentiated by ONE render_adjoint call on every
  schedule; each job's image is compared with the oracle's render of that job alone, and
  the gradients with the sum of the oracle's per-job gradients (the filter angles per job),
  over the pixels whose paths are identical in FP32 and FP64 and whose gradient is well
  conditioned (parity.well_conditioned_pixels: one view has a path refracting near the
  glass sphere's critical angle, whose index derivative has a condition number ~1e5).
* Large: the 500,018-triangle workload at its full size (1024x1024, 128 spp, depth 12, 16
  polarizer angles): sampled pixels of the primal, and the adjoint of a seeded linear loss
  on an 8x8 crop, against the oracle.
"""
import copy

import numpy as np
import pytest

from paper_2607_13265_gb300 import scenegen as sg
from parity import IMG_TOL_P999, GRAD_TOL, image_rel_err, flat, grad_rel, scalar_rel, well_conditioned_pixels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_13265_gb300 import build, api
    build.build()
    return torch, api, api.Context(0), oracle_mod


def _signatures(torch, api, dctx, gs, jobs, P):
    """The jobs' primal image and path signatures; returns a batch of the same jobs WITHOUT
    the signature output (the signature buffer is freed when this returns)."""
    sig = torch.zeros(sum(j.num_paths for j in jobs), dtype=torch.int32, device="cuda")
    img = api.render_primal(dctx, gs, api.pack_jobs(jobs, path_sig=sig), P)
    dctx.sync_status()
    return api.pack_jobs(jobs), img, sig.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("schedule", [(0, 128), (1, 256), (2, 128), (3, 128)],
                         ids=["grid", "persistent", "wavefront", "sweep"])
def test_views_angles_batch_matches_oracle_per_job(env, schedule):
    torch, api, dctx, O = env
    scene, jobs = sg.cornell_views(3, 4, 4, 6, (24, 17, 31))
    plain = copy.copy(jobs[1])
    plain.filter, plain.thetas, plain.stream = sg.FILTER_NONE, [], 9
    jobs.append(plain)
    gs = api.GpuScene(dctx, scene)
    prev = dctx.get_launch()
    dctx.set_launch(*schedule, 0, *schedule, 0)
    try:
        P = api.device_params(scene, api.pack_jobs(jobs))
        batch, img, sig = _signatures(torch, api, dctx, gs, jobs, P)
        views = [v.double().cpu().numpy() for v in api.image_views(batch, img)]
        base = 0
        for j, view in zip(jobs, views):
            o, _, so = O.OracleScene(scene).render(j, scene.params(), paths=True)
            same = sig[base:base + j.num_paths] == so
            base += j.num_paths
            assert same.mean() >= 0.99, same.mean()
            ok = same.reshape(-1, j.spp).all(1)
            err = image_rel_err(flat(view), o)[:, ok]
            assert float(np.quantile(err, 0.999)) <= IMG_TOL_P999
            assert float(err.max()) <= 10 * IMG_TOL_P999

        # adjoint: one call over all jobs against the per-job oracle gradients
        ajobs = api.adjoint_jobs(jobs)
        adj, _, asig = _signatures(torch, api, dctx, gs, ajobs, P)
        rng = np.random.default_rng(17)
        dI, ref, base = [], None, 0
        theta_ref = []
        for j in ajobs:
            _, _, so = O.OracleScene(scene).render(j, scene.params(), paths=True)
            keep = (asig[base:base + j.num_paths] == so).reshape(-1, j.spp).all(1)
            base += j.num_paths
            d = rng.normal(size=(j.num_angles, j.num_pixels, 3, 4)) * keep[None, :, None, None]
            # pixels whose gradient FP32 cannot resolve (condition number above ~1e3) are left out
            d *= well_conditioned_pixels(O, scene, j, d)[None, :, None, None]
            dI.append(d.ravel())
            r = O.OracleScene(scene).gradient(j, scene.params(), d, mode="replay")
            theta_ref.append(r["theta"][:j.num_angles] if j.filter != sg.FILTER_NONE else np.zeros(0))
            ref = r if ref is None else {k: ref[k] + r[k] if k != "theta" else ref[k] for k in ref}
        d_img = torch.as_tensor(np.concatenate(dI), dtype=torch.float32, device="cuda")
        assert d_img.numel() == adj.image_floats
        got = {k: v.double().cpu().numpy() for k, v in api.render_adjoint(dctx, gs, adj, P, d_img).items()}
        dctx.sync_status()
    finally:
        dctx.set_launch(*prev)
    for t, (off, w, h, ch) in enumerate(scene.tex_desc):
        if scene.tex_differentiable[t]:
            o = ref["tex"][off:off + w * h * ch]
            assert np.linalg.norm(o) > 0
            assert grad_rel(got["tex"][off:off + w * h * ch], o) <= GRAD_TOL
    for k in ("ior", "le"):
        assert grad_rel(got[k][:ref[k].size], ref[k]) <= GRAD_TOL, k
        assert float(scalar_rel(got[k][:ref[k].size], ref[k]).max()) <= GRAD_TOL, k
    th = np.concatenate(theta_ref)
    assert got["theta"].size == th.size
    assert grad_rel(got["theta"], th) <= GRAD_TOL
    assert float(scalar_rel(got["theta"], th).max()) <= GRAD_TOL


def test_large_workload_sampled_pixels_and_crop_gradient(env):
    """The large workload at full size: 24 sampled pixels of the primal, and the gradient of a
    nonnegative weighting of the filtered intensities (s0 of every angle's image) on an 8x8
    crop over a mesh.

    FP32 cannot place this workload's texture taps as precisely as FP64: a hit at grazing
    incidence moves along the surface by ~1/cos of its rounding error, so some vertices'
    texture coordinates shift by a fraction of a texel of the 1024^2 maps, moving gradient
    between neighbouring texels although every path is identical.  Measured with the FP64
    oracle alone (its inputs rounded to float32, same paths, this crop and loss): the albedo
    map's gradient moves by 0.56% at full resolution, 0.076% summed over 8x8-texel blocks and
    0.016% over 32x32 blocks; the roughness map's by 0.74%, 0.14% and 0.014%; the scalar
    groups by 2e-5 or less.  So the two maps are compared on 32x32-texel block sums, the
    scalars per group and per element.  A loss with random signs would also make the crop's
    texel sums cancel 10-20x; the nonnegative one does not."""
    torch, api, dctx, O = env
    scene, job = sg.large_scene()
    gs = api.GpuScene(dctx, scene)
    P = api.device_params(scene, api.pack_jobs([job]))
    batch, img, sig = _signatures(torch, api, dctx, gs, [job], P)
    oscene = O.OracleScene(scene)
    # primal: 24 sampled pixels recomputed one by one (all 16 angles)
    pix = np.sort(np.random.default_rng(23).choice(job.num_pixels, 24, replace=False))
    o, _, so = oscene.render(job, scene.params(), pixels=pix, paths=True)
    g = flat(api.image_views(batch, img)[0].double().cpu().numpy())[:, pix]
    # a pixel is compared when all its 128 paths are identical in FP32 and FP64; at depth 12 on
    # 500k displaced triangles about 0.3% of the paths part (a grazing hit on a neighbouring
    # triangle), so about 1 - 0.997^128 = 32% of the pixels hold at least one such path
    same = (sig.reshape(-1, job.spp)[pix].ravel() == so).reshape(-1, job.spp).all(1)
    assert same.mean() >= 0.5, same.mean()
    err = image_rel_err(g, o)[:, same]
    assert float(err.max()) <= 10 * IMG_TOL_P999

    x0, y0 = 480, 560
    crop = np.array([(y0 + dy) * job.width + x0 + dx for dy in range(8) for dx in range(8)], np.int64)
    aj = api.adjoint_jobs([job])
    adj, _, asig = _signatures(torch, api, dctx, gs, aj, P)
    _, _, so = oscene.render(aj[0], scene.params(), pixels=crop, paths=True)
    keep = (asig.reshape(-1, job.spp)[crop].ravel() == so).reshape(-1, job.spp).all(1)
    assert keep.mean() >= 0.5, keep.mean()
    w = np.zeros((job.num_angles, len(crop), 3, 4))
    w[..., 0] = np.random.default_rng(29).uniform(0.5, 1.5, (job.num_angles, len(crop), 3)) * keep[None, :, None]
    W = torch.zeros(adj.image_floats, dtype=torch.float32, device="cuda")
    W.view(job.num_angles, -1, 3, 4)[:, torch.as_tensor(crop, device="cuda")] = torch.as_tensor(
        w, dtype=torch.float32, device="cuda")
    got = {k: v.double().cpu().numpy() for k, v in api.render_adjoint(dctx, gs, adj, P, W).items()}
    dctx.sync_status()
    ref = oscene.gradient(aj[0], scene.params(), w, pixels=crop, mode="replay")
    for t in (0, 1):
        off, tw, th, ch = scene.tex_desc[t]
        blocks = lambda x: x[off:off + tw * th * ch].reshape(th // 32, 32, tw // 32, 32, ch).sum((1, 3))
        assert np.linalg.norm(blocks(ref["tex"])) > 0, t
        assert grad_rel(blocks(got["tex"]), blocks(ref["tex"])) <= GRAD_TOL, (t, grad_rel(blocks(got["tex"]),
                                                                                       blocks(ref["tex"])))
    for k in ("ior", "le", "sheet", "theta"):
        o = ref[k]
        if np.linalg.norm(o) == 0:
            continue
        assert grad_rel(got[k][:o.size], o) <= GRAD_TOL, k
        assert float(scalar_rel(got[k][:o.size], o).max()) <= GRAD_TOL, (k, got[k][:o.size], o)


def test_views_angles_full_size_sampled_pixels(env):
    """The views x angles workload at its full size (8 views 128^2..512^2, 64 angles, 16 spp,
    depth 8) in the launch configuration the benchmark's autotuner picks for it (grid primal,
    wavefront adjoint): the adjoint's 15.1 M paths fill four waves shared by the views, the
    larger views split between waves.  Sampled pixels of every view against the oracle, for
    the image and for the gradient of a linear loss on those pixels."""
    torch, api, dctx, O = env
    scene, jobs = sg.cornell_views(8, 64, 16, 8)
    gs = api.GpuScene(dctx, scene)
    prev = dctx.get_launch()
    dctx.set_launch(0, 256, 0, 2, 128, 0, 0)
    rng = np.random.default_rng(41)
    try:
        P = api.device_params(scene, api.pack_jobs(jobs))
        batch, img, sig = _signatures(torch, api, dctx, gs, jobs, P)
        views = api.image_views(batch, img)
        base = 0
        for j, view in zip(jobs, views):
            pix = np.sort(rng.choice(j.num_pixels, 6, replace=False))
            o, _, so = O.OracleScene(scene).render(j, scene.params(), pixels=pix, paths=True)
            same = (sig[base:base + j.num_paths].reshape(-1, j.spp)[pix].ravel() == so).reshape(-1, j.spp).all(1)
            base += j.num_paths
            g = flat(view.double().cpu().numpy())[:, pix]
            err = image_rel_err(g, o)[:, same]
            assert same.mean() >= 0.5 and float(err.max()) <= 10 * IMG_TOL_P999
        ajobs = api.adjoint_jobs(jobs)
        adj, _, asig = _signatures(torch, api, dctx, gs, ajobs, P)
        W = torch.zeros(adj.image_floats, dtype=torch.float32, device="cuda")
        ref, theta_ref, base = None, [], 0
        for j, off in zip(ajobs, adj.offsets):
            pix = np.sort(rng.choice(j.num_pixels, 4, replace=False))
            _, _, so = O.OracleScene(scene).render(j, scene.params(), pixels=pix, paths=True)
            keep = (asig[base:base + j.num_paths].reshape(-1, j.spp)[pix].ravel() == so).reshape(-1, j.spp).all(1)
            base += j.num_paths
            w = rng.normal(size=(j.num_angles, len(pix), 3, 4)) * keep[None, :, None, None]
            full = np.zeros((j.num_angles, j.num_pixels, 3, 4))
            full[:, pix] = w
            full *= well_conditioned_pixels(O, scene, j, full)[None, :, None, None]
            W[off:off + full.size] = torch.as_tensor(full.ravel(), dtype=torch.float32, device="cuda")
            r = O.OracleScene(scene).gradient(j, scene.params(), full[:, pix], pixels=pix, mode="replay")
            theta_ref.append(r["theta"][:j.num_angles])
            ref = r if ref is None else {k: ref[k] + r[k] if k != "theta" else ref[k] for k in ref}
        got = {k: v.double().cpu().numpy() for k, v in api.render_adjoint(dctx, gs, adj, P, W).items()}
        dctx.sync_status()
    finally:
        dctx.set_launch(*prev)
    off, tw, th, ch = scene.tex_desc[3]
    assert grad_rel(got["tex"][off:off + tw * th * ch], ref["tex"][off:off + tw * th * ch]) <= GRAD_TOL
    for k in ("ior", "le"):
        assert grad_rel(got[k][:ref[k].size], ref[k]) <= GRAD_TOL, k
    assert grad_rel(got["theta"], np.concatenate(theta_ref)) <= GRAD_TOL
