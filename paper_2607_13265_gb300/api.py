"""Python binding of the C ABI: contexts, scenes, render_primal / render_adjoint and
the torch.autograd.Function that puts render_adjoint behind backward().

PyTorch only provides device memory and streams here; every step of the path
runs in the CUDA library.  Names follow the paper: the primal image I(pi), its
adjoint dg/dI and the parameter gradient dg/dpi (Sec. 3.1, Eq. 1).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from .scenegen import FILTER_NONE


def _check(ctx_handle, status: int, what: str):
    if status != L.DPPT_OK:
        msg = L.load().dppt_last_error(ctx_handle)
        raise L.DpptError(f"{what} failed ({L.STATUS_NAMES.get(status, status)}): "
                          f"{msg.decode() if msg else ''}")


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr()) if t.numel() > 0 else None
    return t


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A dppt context on one CUDA device (owns its workspace and status word)."""

    def __init__(self, device: int = 0):
        self.lib = L.load()
        self.device = device
        h = ctypes.c_void_p()
        st = self.lib.dppt_create(ctypes.byref(h), device)
        if st != L.DPPT_OK:
            raise L.DpptError(f"dppt_create failed ({L.STATUS_NAMES.get(st, st)})")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.dppt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_launch(self, schedule: int, block_size: int, blocks_per_sm: int = 0, adj_schedule: int | None = None,
                   adj_block_size: int | None = None, adj_blocks_per_sm: int | None = None,
                   adj_scatter: int | None = None):
        """Launch shape of render_primal (and of render_adjoint; same as the primal unless given).
        adj_scatter: 0 texel gradients combined per warp group, 1 one atomic per lane (unchanged
        when None)."""
        l = L.Launch(schedule, block_size, blocks_per_sm,
                     schedule if adj_schedule is None else adj_schedule,
                     block_size if adj_block_size is None else adj_block_size,
                     blocks_per_sm if adj_blocks_per_sm is None else adj_blocks_per_sm,
                     self.get_launch()[6] if adj_scatter is None else adj_scatter)
        _check(self.h, self.lib.dppt_set_launch(self.h, ctypes.byref(l)), "dppt_set_launch")

    def get_launch(self) -> tuple:
        """(schedule, block, blocks_per_sm, adj_schedule, adj_block, adj_blocks_per_sm, adj_scatter)"""
        l = L.Launch()
        _check(self.h, self.lib.dppt_get_launch(self.h, ctypes.byref(l)), "dppt_get_launch")
        return (l.schedule, l.block_size, l.blocks_per_sm, l.adj_schedule, l.adj_block_size, l.adj_blocks_per_sm,
                l.adj_scatter)

    def set_replay(self, checkpoint_interval: int = 1, gamma: float = 0.0, eps: float = float("inf"),
                   method: str = "cached", sigma: float = 0.0):
        """Suffix replay of render_adjoint: checkpoint_interval 1 caches every vertex's suffix
        (Sec. 4.3); 4, 8 or 16 is the hybrid cached replay of Sec. 4.4 with thresholds gamma
        (depolarization index, scalar route) and eps (|det|, inversion route).  method 'pprb'
        selects the basic polarized PRB baseline with diagonal noise of deviation sigma."""
        r = L.Replay({"cached": 0, "pprb": 1}[method], int(checkpoint_interval), float(gamma), float(eps), float(sigma))
        _check(self.h, self.lib.dppt_set_replay(self.h, ctypes.byref(r)), "dppt_set_replay")

    def get_replay(self) -> tuple:
        """(checkpoint_interval, gamma, eps, method, sigma)"""
        r = L.Replay()
        _check(self.h, self.lib.dppt_get_replay(self.h, ctypes.byref(r)), "dppt_get_replay")
        return (r.checkpoint_interval, r.gamma, r.eps, ("cached", "pprb")[r.method], r.sigma)

    def adjoint_footprint(self, max_depth: int) -> dict:
        out = (ctypes.c_int64 * 4)()
        _check(self.h, self.lib.dppt_adjoint_footprint(self.h, max_depth, out), "dppt_adjoint_footprint")
        return {"local_bytes_per_thread": out[0], "registers": out[1], "threads_per_sm": out[2], "sms": out[3]}

    STAGES = ("primal", "adjoint", "wf_init", "wf_extend", "wf_shade", "wf_shadow", "wf_cache", "wf_replay",
              "wf_sweep", "wf_pixels", "filter")

    def stage_stats(self, timing: bool = False, reset: bool = True) -> dict:
        """{stage: (launches, ms)} since the last reset; then switches event timing on/off."""
        n = (ctypes.c_int64 * 16)()
        ms = (ctypes.c_double * 16)()
        _check(self.h, self.lib.dppt_stage_stats(self.h, int(timing), int(reset), n, ms), "dppt_stage_stats")
        return {name: (int(n[k]), float(ms[k])) for k, name in enumerate(self.STAGES)}

    def query_workspace(self, batch: "JobBatch") -> int:
        b = ctypes.c_size_t()
        _check(self.h, self.lib.dppt_query_workspace(self.h, batch.c_jobs, batch.n, ctypes.byref(b)),
               "dppt_query_workspace")
        return int(b.value)

    def sync_status(self, stream=None):
        _check(self.h, self.lib.dppt_sync_status(self.h, _stream_ptr(stream)), "dppt_sync_status")


class GpuScene:
    """A scene uploaded to the device (BVH built by the library at upload)."""

    def __init__(self, ctx: Context, scene):
        self.ctx = ctx
        self.scene = scene
        keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dt)
            keep.append(a)
            return a

        verts = arr(scene.verts, np.float32)
        uvs = arr(scene.uvs, np.float32)
        tris = arr(scene.tris, np.int32)
        tmat = arr(scene.tri_mat, np.int32)
        tlight = arr(scene.tri_light, np.int32)
        sph = arr(scene.spheres, np.float32)
        smat = arr(scene.sph_mat, np.int32)
        mats = (L.Material * len(scene.materials))()
        for i, m in enumerate(scene.materials):
            mats[i] = L.Material(m.type, m.albedo_tex, m.rough_tex, m.ior_index, m.sheet_index, m.normal_tex,
                                 m.eta_re, m.eta_im,
                                 (ctypes.c_float * 3)(*m.t1), (ctypes.c_float * 3)(*m.t2), m.retard, m.emission)
        lights = arr(scene.lights, np.float32)
        texd = arr(scene.tex_desc, np.int64)
        cams = arr(scene.cameras, np.float32)
        p = scene.params()
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a.size else None
        d = L.SceneDesc(len(verts), P(verts), P(uvs), len(tris), P(tris), P(tmat), P(tlight),
                        len(sph), P(sph), P(smat), len(scene.materials), ctypes.cast(mats, ctypes.c_void_p),
                        len(lights), P(lights), len(texd), P(texd), int(p["tex"].size),
                        len(cams), P(cams), len(scene.ior), len(scene.sheet), float(scene.ray_eps()))
        h = ctypes.c_void_p()
        _check(ctx.h, ctx.lib.dppt_scene_upload(ctx.h, ctypes.byref(d), ctypes.byref(h)), "dppt_scene_upload")
        self.h = h
        del keep

    def info(self) -> dict:
        out = (ctypes.c_int64 * 5)()
        _check(self.ctx.h, self.ctx.lib.dppt_scene_info(self.h, out), "dppt_scene_info")
        return {"bvh_nodes": out[0], "triangles": out[1], "spheres": out[2], "device_bytes": out[3], "bvh_depth": out[4]}

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.dppt_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class JobBatch:
    """Jobs packed for the C ABI, with image offsets and the filter-angle vector."""
    jobs: list
    c_jobs: object
    offsets: list
    image_floats: int
    theta: np.ndarray

    @property
    def n(self) -> int:
        return len(self.jobs)


def pack_jobs(jobs, path_sig: torch.Tensor | None = None) -> JobBatch:
    """Lay the jobs' images out back to back and collect their filter angles.  A job seen
    through a camera filter needs at least one angle: with none, the angle offsets of the
    later jobs would no longer match the angle vector."""
    arr = (L.Job * len(jobs))()
    off, toff, offsets, thetas = 0, 0, [], []
    sig_off = 0
    for i, j in enumerate(jobs):
        if j.filter != FILTER_NONE and len(j.thetas) == 0:
            raise ValueError(f"job {i}: a camera filter needs at least one angle")
        nang = j.num_angles
        arr[i] = L.Job(j.camera, j.width, j.height, j.spp, j.max_depth, j.filter,
                       nang if j.filter != FILTER_NONE else 1, toff if j.filter != FILTER_NONE else 0,
                       j.seed, j.stream, j.pass_id, 0, off, None)
        if path_sig is not None:
            arr[i].path_sig = path_sig.data_ptr() + 4 * sig_off
            sig_off += j.num_paths
        offsets.append(off)
        off += nang * j.width * j.height * 12
        if j.filter != FILTER_NONE:
            thetas += list(j.thetas)
            toff += nang
    return JobBatch(list(jobs), arr, offsets, off, np.array(thetas if thetas else [0.0], np.float64))


def device_params(scene, batch: JobBatch | None = None, params: dict | None = None, device="cuda") -> dict:
    """Float32 device copies of the differentiable parameters {tex, ior, le, sheet, theta}."""
    p = dict(scene.params() if params is None else params)
    out = {k: torch.as_tensor(np.asarray(p[k], np.float64).ravel(), dtype=torch.float32, device=device)
           for k in ("tex", "ior", "le", "sheet")}
    th = p.get("theta", batch.theta if batch is not None else np.zeros(1))
    out["theta"] = torch.as_tensor(np.asarray(th, np.float64).ravel(), dtype=torch.float32, device=device)
    return out


def _c_params(p: dict) -> L.Params:
    return L.Params(_ptr(p["tex"]), _ptr(p["ior"]), _ptr(p["le"]), _ptr(p["sheet"]), _ptr(p["theta"]))


def render_primal(ctx: Context, gs: GpuScene, batch: JobBatch, params: dict, image: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """Phase 1: the primal Stokes images of all jobs (one megakernel launch per depth bucket, or the
    wavefront's stage kernels, by the context's schedule)."""
    if image is None:
        image = torch.empty(batch.image_floats, dtype=torch.float32, device=params["tex"].device)
    cp = _c_params(params)
    _check(ctx.h, ctx.lib.dppt_render_primal(ctx.h, gs.h, batch.c_jobs, batch.n, ctypes.byref(cp), _ptr(image),
                                             _stream_ptr(stream)), "dppt_render_primal")
    return image


WORK_KEYS = ("paths", "vertices", "rays", "shadow_rays", "nodes", "shadow_nodes", "tri_tests", "shadow_tri_tests",
             "sph_tests", "shadow_sph_tests")


def count_work(ctx: Context, gs: GpuScene, batch: JobBatch, params: dict) -> dict:
    """Work units of the jobs' paths (instrumented primal on the same BVH; untimed)."""
    out = (ctypes.c_uint64 * 10)()
    cp = _c_params(params)
    _check(ctx.h, ctx.lib.dppt_count_work(ctx.h, gs.h, batch.c_jobs, batch.n, ctypes.byref(cp), out),
           "dppt_count_work")
    return dict(zip(WORK_KEYS, [int(x) for x in out]))


SCHEDULE_NAMES = {0: "grid", 1: "persistent", 2: "wavefront", 3: "sweep"}


def autotune(ctx: Context, gs: GpuScene, batch: JobBatch, params: dict, reps: int = 2) -> dict:
    """Run the library's autotuner on these jobs; the context keeps the fastest shapes."""
    best = L.Launch()
    times = (ctypes.c_float * 24)()
    cp = _c_params(params)
    _check(ctx.h, ctx.lib.dppt_autotune(ctx.h, gs.h, batch.c_jobs, batch.n, ctypes.byref(cp), reps,
                                        ctypes.byref(best), times), "dppt_autotune")
    table = {}
    for si in range(4):
        for bi, b in enumerate((64, 128, 256)):
            k = 3 * si + bi
            table[f"{SCHEDULE_NAMES[si]}/{b}"] = {"primal_ms": times[2 * k], "adjoint_ms": times[2 * k + 1]}
    return {"primal": (SCHEDULE_NAMES[best.schedule], best.block_size),
            "adjoint": (SCHEDULE_NAMES[best.adj_schedule], best.adj_block_size),
            "adjoint_scatter": ("warp", "lane")[best.adj_scatter], "times_ms": table}


def zero_grads(params: dict) -> dict:
    return {k: torch.zeros_like(v) for k, v in params.items()}


def render_adjoint(ctx: Context, gs: GpuScene, batch: JobBatch, params: dict, d_image: torch.Tensor,
                   grads: dict | None = None, stream=None) -> dict:
    """Phases 2+3 (cached suffix replay): ADDS dg/dpi into `grads` and returns it."""
    if grads is None:
        grads = zero_grads(params)
    cp = _c_params(params)
    cg = L.Grads(_ptr(grads.get("tex")), _ptr(grads.get("ior")), _ptr(grads.get("le")), _ptr(grads.get("sheet")),
                 _ptr(grads.get("theta")))
    _check(ctx.h, ctx.lib.dppt_render_adjoint(ctx.h, gs.h, batch.c_jobs, batch.n, ctypes.byref(cp), _ptr(d_image),
                                              ctypes.byref(cg), _stream_ptr(stream)), "dppt_render_adjoint")
    return grads


def raw_batch(batch: JobBatch) -> JobBatch:
    """The batch's jobs without their camera filter: render_primal of this batch writes each
    job's raw (unfiltered) image [H][W][3][4], back to back; the paths are the same."""
    import copy
    jobs = []
    for j in batch.jobs:
        k = copy.copy(j)
        k.filter, k.thetas = FILTER_NONE, []
        jobs.append(k)
    return pack_jobs(jobs)


def loss_l2(ctx: Context, gs: GpuScene, batch: JobBatch, params: dict, raw: torch.Tensor, raw_offsets,
            target: torch.Tensor, scale: float, loss: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """scale * sum |C(theta_a) raw - T_a|^2 over the batch's jobs, angles and pixels (device double)."""
    if loss is None:
        loss = torch.empty((), dtype=torch.float64, device=raw.device)
    cp = _c_params(params)
    offs = np.ascontiguousarray(raw_offsets, np.int64)
    _check(ctx.h, ctx.lib.dppt_loss_l2(ctx.h, gs.h, batch.c_jobs, batch.n, ctypes.byref(cp), _ptr(raw),
                                       offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(target),
                                       float(scale), _ptr(loss), _stream_ptr(stream)), "dppt_loss_l2")
    return loss


def render_adjoint_l2(ctx: Context, gs: GpuScene, batch: JobBatch, params: dict, raw: torch.Tensor, raw_offsets,
                      target: torch.Tensor, scale: float, grads: dict | None = None, stream=None) -> dict:
    """render_adjoint with the adjoint input of the fused L2 loss formed per pixel: ADDS
    the gradient of scale * sum |C_a raw - T_a|^2 into `grads` and returns it."""
    if grads is None:
        grads = zero_grads(params)
    cp = _c_params(params)
    cg = L.Grads(_ptr(grads.get("tex")), _ptr(grads.get("ior")), _ptr(grads.get("le")), _ptr(grads.get("sheet")),
                 _ptr(grads.get("theta")))
    offs = np.ascontiguousarray(raw_offsets, np.int64)
    _check(ctx.h, ctx.lib.dppt_render_adjoint_l2(ctx.h, gs.h, batch.c_jobs, batch.n, ctypes.byref(cp), _ptr(raw),
                                                 offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _ptr(target),
                                                 float(scale), ctypes.byref(cg), _stream_ptr(stream)),
           "dppt_render_adjoint_l2")
    return grads


def image_views(batch: JobBatch, image: torch.Tensor) -> list:
    """Per-job views [angles][H][W][3][4] of a packed image buffer."""
    out = []
    for j, off in zip(batch.jobs, batch.offsets):
        n = j.num_angles * j.width * j.height * 12
        out.append(image[off:off + n].view(j.num_angles, j.height, j.width, 3, 4))
    return out


class PolarizedRender(torch.autograd.Function):
    """I = render(pi) with dI^T-vector products from render_adjoint (cached suffix replay).

    forward(ctx_obj, gscene, batch, adjoint_batch, tex, ior, le, sheet, theta) -> packed image.
    The adjoint uses `adjoint_batch` (same jobs with a different pass id: decorrelated
    paths, PRB phase 2) so that the gradient estimate is independent of the image."""

    @staticmethod
    def forward(fctx, dctx, gs, batch, adj_batch, tex, ior, le, sheet, theta):
        params = {"tex": tex.detach(), "ior": ior.detach(), "le": le.detach(), "sheet": sheet.detach(),
                  "theta": theta.detach()}
        image = render_primal(dctx, gs, batch, params)
        fctx.dctx, fctx.gs, fctx.adj_batch = dctx, gs, adj_batch
        fctx.save_for_backward(tex, ior, le, sheet, theta)
        return image

    @staticmethod
    def backward(fctx, d_image):
        tex, ior, le, sheet, theta = fctx.saved_tensors
        params = {"tex": tex.detach(), "ior": ior.detach(), "le": le.detach(), "sheet": sheet.detach(),
                  "theta": theta.detach()}
        grads = render_adjoint(fctx.dctx, fctx.gs, fctx.adj_batch, params, d_image.contiguous())
        return (None, None, None, None, grads["tex"], grads["ior"], grads["le"], grads["sheet"], grads["theta"])


class PolarizedL2(torch.autograd.Function):
    """mean((I(pi) - T)^2) over all jobs and angles, fused into the camera filter: the
    forward keeps only the raw image (12 floats per pixel, whatever the number of angles)
    and the backward forms the adjoint input per pixel (dppt_render_adjoint_l2).

    forward(ctx_obj, gscene, batch, adjoint_batch, target, tex, ior, le, sheet, theta) -> loss."""

    @staticmethod
    def forward(fctx, dctx, gs, batch, adj_batch, target, tex, ior, le, sheet, theta):
        params = {"tex": tex.detach(), "ior": ior.detach(), "le": le.detach(), "sheet": sheet.detach(),
                  "theta": theta.detach()}
        rb = raw_batch(batch)
        raw = render_primal(dctx, gs, rb, params)
        n = target.numel()
        loss = loss_l2(dctx, gs, batch, params, raw, rb.offsets, target, 1.0 / n)
        fctx.dctx, fctx.gs, fctx.adj_batch, fctx.raw_offsets, fctx.n = dctx, gs, adj_batch, rb.offsets, n
        fctx.save_for_backward(tex, ior, le, sheet, theta, raw, target)
        return loss.to(torch.float32)

    @staticmethod
    def backward(fctx, g):
        tex, ior, le, sheet, theta, raw, target = fctx.saved_tensors
        params = {"tex": tex.detach(), "ior": ior.detach(), "le": le.detach(), "sheet": sheet.detach(),
                  "theta": theta.detach()}
        grads = render_adjoint_l2(fctx.dctx, fctx.gs, fctx.adj_batch, params, raw, fctx.raw_offsets, target,
                                  1.0 / fctx.n)
        for v in grads.values():
            v.mul_(g)
        return (None, None, None, None, None, grads["tex"], grads["ior"], grads["le"], grads["sheet"], grads["theta"])


class ImageL2(torch.autograd.Function):
    """mean((I - T)^2) without image-sized temporaries in the forward; the backward
    returns dg/dI = 2 (I - T) / N, the adjoint image render_adjoint consumes."""

    @staticmethod
    def forward(fctx, img, target):
        fctx.save_for_backward(img, target)
        acc = torch.zeros((), dtype=torch.float64, device=img.device)
        step = 1 << 24
        for c in range(0, img.numel(), step):
            d = img[c:c + step] - target[c:c + step]
            acc += (d * d).sum(dtype=torch.float64)
        return (acc / img.numel()).to(img.dtype)

    @staticmethod
    def backward(fctx, g):
        img, target = fctx.saved_tensors
        return torch.sub(img, target).mul_(2.0 / img.numel()).mul_(g), None


def adjoint_jobs(jobs, pass_id: int = 1):
    """Copies of the jobs with another pass id (decorrelated paths for the adjoint)."""
    import copy
    out = []
    for j in jobs:
        k = copy.copy(j)
        k.pass_id = pass_id
        out.append(k)
    return out


def radians(deg) -> float:
    return math.radians(deg)
