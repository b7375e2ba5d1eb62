"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64 oracle on
the same seeded jobs and compare them.

Image metric (the per-pixel relative error of the Stokes image): for pixel p,
channel c and Stokes component k,
    e = |g - o| / max(|o_{c,s0}|, 1e-3 * mean_p |o_{c,s0}|)
i.e. every component is measured against the intensity of its pixel and channel
(|s_k| <= s0 for any physical Stokes vector), with a floor for black pixels.
Gradient metric: ||g - o||_2 / ||o||_2 per parameter group, and for the scalar groups
(indices of refraction, emitter Stokes vectors, sheet and filter angles) also per element,
|g_i - o_i| / max(|o_i|, 1e-2 max_j |o_j|): an element below 1% of its group's largest is
measured at that scale, since its FP32 sum cancels terms of the group's size.
"""
from __future__ import annotations

import numpy as np

IMG_TOL_P999 = 1e-4
GRAD_TOL = 1e-3


def image_rel_err(g: np.ndarray, o: np.ndarray) -> np.ndarray:
    """g, o: [..., npix, 3, 4] -> relative errors of the same shape."""
    s0 = np.abs(o[..., :1])
    floor = 1e-3 * max(float(np.abs(o[..., 0]).mean()), 1e-30)
    return np.abs(g - o) / np.maximum(s0, floor)


def gpu_image(api, dctx, gs, jobs, params_np=None, scene=None, with_sig=False):
    import torch
    sig = None
    if with_sig:
        sig = torch.zeros(sum(j.num_paths for j in jobs), dtype=torch.int32, device="cuda")
    batch = api.pack_jobs(jobs, path_sig=sig)
    P = api.device_params(scene or gs.scene, batch, params_np)
    img = api.render_primal(dctx, gs, batch, P)
    dctx.sync_status()
    views = [v.double().cpu().numpy() for v in api.image_views(batch, img)]
    if with_sig:
        return views, sig.cpu().numpy().view(np.uint32), batch, P
    return views, batch, P


def flat(view: np.ndarray) -> np.ndarray:
    """[A][H][W][3][4] -> [A][H*W][3][4]"""
    a, h, w = view.shape[:3]
    return view.reshape(a, h * w, 3, 4)


def grad_rel(g: np.ndarray, o: np.ndarray) -> float:
    n = np.linalg.norm(o)
    return float(np.linalg.norm(g - o) / n) if n > 0 else float(np.linalg.norm(g))


def scalar_rel(g: np.ndarray, o: np.ndarray) -> np.ndarray:
    """Per-element relative errors of a scalar gradient group (see the module docstring)."""
    g, o = np.asarray(g, np.float64), np.asarray(o, np.float64)
    floor = 1e-2 * float(np.abs(o).max()) if o.size else 0.0
    return np.abs(g - o) / np.maximum(np.abs(o), max(floor, 1e-300))


def float32_inputs(scene):
    """A copy of the scene whose geometry, cameras, lights, textures and indices are rounded
    to float32: the inputs the GPU library actually receives."""
    import copy
    f32 = lambda a: np.asarray(a, np.float64).astype(np.float32).astype(np.float64)
    s = copy.deepcopy(scene)
    s._verts = [f32(v) for v in s._verts]
    s._uvs = [f32(v) for v in s._uvs]
    s.spheres = f32(s.spheres)
    s._lights = [f32(v) for v in s._lights]
    s._cameras = [f32(v) for v in s._cameras]
    s._tex_blocks = [f32(v) for v in s._tex_blocks]
    s._le = [f32(v) for v in s._le]
    s.ior = [float(np.float32(x)) for x in s.ior]
    s.sheet = [float(np.float32(x)) for x in s.sheet]
    s.eps = float(np.float32(scene.ray_eps()))
    return s


def well_conditioned_pixels(oracle_mod, scene, job, dI, rel: float = 6e-5) -> np.ndarray:
    """Pixels whose FP64 gradient moves by at most `rel` (relative, per parameter group's
    largest element) when the scene's inputs are rounded to float32.  That rounding is a
    relative perturbation of ~6e-8, so a larger move means a condition number above ~1e3:
    FP32 arithmetic, whose rounding perturbs every step by the same order, cannot then
    resolve the pixel's gradient to 1e-3.  This happens for paths that refract near the
    critical angle (the index-of-refraction derivative carries 1/cos(theta_t)).  Only
    pixels with a nonzero adjoint are examined; dI is [angles][pixels][3][4]."""
    import copy
    o64 = oracle_mod.OracleScene(scene)
    s32 = float32_inputs(scene)
    o32 = oracle_mod.OracleScene(s32)
    j32 = copy.copy(job)
    if job.thetas:
        j32.thetas = [float(np.float32(t)) for t in job.thetas]
    ok = np.ones(dI.shape[1], bool)
    for p in np.nonzero(np.abs(dI).reshape(dI.shape[0], dI.shape[1], -1).max((0, 2)) > 0)[0]:
        g64 = o64.gradient(job, scene.params(), dI[:, p:p + 1], pixels=[p], mode="replay")
        g32 = o32.gradient(j32, s32.params(), dI[:, p:p + 1], pixels=[p], mode="replay")
        for k in g64:
            a, b = np.asarray(g64[k]), np.asarray(g32[k])
            if a.size and np.abs(a - b).max() > rel * max(np.abs(a).max(), 1e-12):
                ok[p] = False
    return ok


def image_input_sensitivity(oracle_mod, scene, job, pixels) -> np.ndarray:
    """Per pixel of `pixels`: how far the FP64 image moves (largest Stokes component, in the
    image_rel_err metric) when the scene's inputs are rounded to float32.  That rounding
    perturbs the inputs by ~6e-8 relative, and an FP32 hit point carries an error of the same
    order, so the move measures how much of an FP32 program's error the pixel's own
    conditioning explains: a move above 1e-5 means a condition number above ~150, where FP32
    cannot resolve the pixel to 1e-4.  Large moves come where a white-noise texture
    (neighbouring texels independent) sets the roughness of a narrow GGX lobe: a 1e-7 shift of
    the hit point changes alpha by ~1e-4 relative and the lobe's tail by up to 1e-3."""
    import copy
    pixels = np.asarray(pixels, np.int64)
    o64, _, _ = oracle_mod.OracleScene(scene).render(job, scene.params(), pixels=pixels, paths=True)
    s32 = float32_inputs(scene)
    j32 = copy.copy(job)
    if job.thetas:
        j32.thetas = [float(np.float32(t)) for t in job.thetas]
    o32, _, _ = oracle_mod.OracleScene(s32).render(j32, s32.params(), pixels=pixels, paths=True)
    return image_rel_err(o32, o64).max(axis=(0, 2, 3))


def identical_path_pixels(api, dctx, gs, job, oracle_scene, params_np):
    """Signatures of the job's paths (its own pass id) on both sides: returns the fraction
    of identical paths and a per-pixel mask of the pixels whose paths are all identical.
    A path whose FP32 and FP64 walks part (a grazing ray on a neighbouring triangle after
    many bounces) is a different sample, not a wrong one: comparisons use the mask."""
    import torch
    sig = torch.zeros(job.num_paths, dtype=torch.int32, device="cuda")
    batch = api.pack_jobs([job], path_sig=sig)
    P = api.device_params(gs.scene, batch, params_np)
    api.render_primal(dctx, gs, batch, P)
    dctx.sync_status()
    sg = sig.cpu().numpy().view(np.uint32)
    _, _, so = oracle_scene.render(job, params_np if params_np is not None else gs.scene.params(), paths=True)
    same = sg == so
    return float(same.mean()), same.reshape(-1, job.spp).all(1)
