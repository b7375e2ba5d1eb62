"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64 oracle on
the same seeded jobs and compare them.

Image metric (the per-pixel relative error of the Stokes image): for pixel p,
channel c and Stokes component k,
    e = |g - o| / max(|o_{c,s0}|, 1e-3 * mean_p |o_{c,s0}|)
i.e. every component is measured against the intensity of its pixel and channel
(|s_k| <= s0 for any physical Stokes vector), with a floor for black pixels.
Gradient metric: ||g - o||_2 / ||o||_2 per parameter group.
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
