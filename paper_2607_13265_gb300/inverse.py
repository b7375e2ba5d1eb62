"""Inverse rendering with Adam on the large workload (Eq. 1: pi* = argmin g(I(pi))).

Scene: 10 displaced meshes of 50,000 triangles (500k), mixed diffuse / rough conductor /
rough dielectric pBRDFs, 3 polarizer sheets and 1 retarder sheet, 4 unpolarized quad
lights; 1024x1024, 128 spp, depth 12, camera polarizer at 16 angles (folded exactly).
Parameters: the 1024^2x3 albedo and 1024^2 roughness textures, optimized with Adam (lr
1e-2) toward a target rendered from seeded target textures with other random numbers.
Each iteration is the fused loss PolarizedL2 (render_primal of the raw image + the loss
folded into the camera filter) + loss.backward() (render_adjoint_l2, cached suffix replay)
+ Adam; --image-loss uses PolarizedRender and mean((I - T)^2) instead.  Prints one JSON line.

  python -m paper_2607_13265_gb300.inverse [--iters 10] [--width 1024] [--spp 128]
"""
from __future__ import annotations

import argparse
import copy
import json
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--lr", type=float, default=1e-2)
    ap.add_argument("--width", type=int, default=1024)
    ap.add_argument("--spp", type=int, default=128)
    ap.add_argument("--depth", type=int, default=12)
    ap.add_argument("--angles", type=int, default=16)
    ap.add_argument("--meshes", type=int, default=10)
    ap.add_argument("--freq", type=int, default=50)
    ap.add_argument("--tex", type=int, default=1024)
    ap.add_argument("--image-loss", action="store_true",
                    help="PolarizedRender + mean((I - T)^2) instead of the fused PolarizedL2")
    args = ap.parse_args(argv)

    import torch
    from . import api, build, scenegen as sg
    build.build()
    t0 = time.time()
    scene, job = sg.large_scene(args.meshes, args.freq, args.tex, args.width, args.spp, args.depth, args.angles)
    t_scene = time.time() - t0
    dctx = api.Context(0)
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    adj = api.pack_jobs(api.adjoint_jobs([job]))
    P = api.device_params(scene, batch)

    # schedule and block size from the autotuner on a reduced copy of the job
    proxy = copy.copy(job)
    proxy.width = proxy.height = max(64, args.width // 4)
    proxy.spp = max(4, args.spp // 8)
    pb = api.pack_jobs(api.adjoint_jobs([proxy]))
    tuning = api.autotune(dctx, gs, pb, api.device_params(scene, pb), reps=1)

    # seeded target textures and image (other random numbers than the optimization's)
    tgt = scene.params()
    (a_off, aw, ah, ach), (r_off, rw, rh, _) = scene.tex_desc[0], scene.tex_desc[1]
    tgt["tex"][a_off:a_off + aw * ah * ach] = sg.smooth_texture(aw, 0.2, 0.9, 30, ach).ravel()
    tgt["tex"][r_off:r_off + rw * rh] = sg.smooth_texture(rw, 0.05, 0.5, 31).ravel()
    tjob = copy.copy(job)
    tjob.seed = 4242
    target = api.render_primal(dctx, gs, api.pack_jobs([tjob]), api.device_params(scene, batch, tgt)).clone()
    target_tex = torch.as_tensor(tgt["tex"], dtype=torch.float32, device="cuda")

    tex = P["tex"].clone().requires_grad_(True)
    others = {k: P[k] for k in ("ior", "le", "sheet", "theta")}
    opt = torch.optim.Adam([tex], lr=args.lr)
    alb = slice(a_off, a_off + aw * ah * ach)
    rough = slice(r_off, r_off + rw * rh)

    def rmse(sl):
        return float(((tex.detach()[sl] - target_tex[sl]) ** 2).mean().sqrt())

    history = []
    times = []
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    mem0 = torch.cuda.memory_allocated()
    rmse0 = {"albedo": rmse(alb), "roughness": rmse(rough)}
    for it in range(args.iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        opt.zero_grad(set_to_none=True)
        adj_it = api.pack_jobs(api.adjoint_jobs([job], pass_id=1 + 2 * it))   # fresh decorrelated paths
        if args.image_loss:
            img = api.PolarizedRender.apply(dctx, gs, batch, adj_it, tex, others["ior"], others["le"],
                                            others["sheet"], others["theta"])
            loss = ((img - target) ** 2).mean()
        else:
            loss = api.PolarizedL2.apply(dctx, gs, batch, adj_it, target, tex, others["ior"], others["le"],
                                         others["sheet"], others["theta"])
        loss.backward()
        opt.step()
        with torch.no_grad():
            tex[alb].clamp_(0.0, 1.0)
            tex[rough].clamp_(0.02, 1.0)
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
        history.append(float(loss))
        job.seed += 1                      # new primal paths each iteration
        batch = api.pack_jobs([job])
    dctx.sync_status()
    paths = 2 * job.num_paths
    lc = dctx.get_launch()
    out = {
        "workload": f"large{args.meshes}x{20 * args.freq ** 2}tris_{args.width}^2_{args.spp}spp_depth{args.depth}_{args.angles}angles",
        "triangles": int(scene.num_triangles), "scene_build_s": t_scene,
        "schedule": {"primal": [api.SCHEDULE_NAMES[lc[0]], lc[1]], "adjoint": [api.SCHEDULE_NAMES[lc[3]], lc[4]]},
        "iterations": args.iters, "ms_per_iteration": times, "median_ms": float(np.median(times)),
        "paths_per_iteration": paths, "paths_per_s": paths / (float(np.median(times)) / 1000.0),
        "loss": history, "texture_rmse_before": rmse0,
        "texture_rmse_after": {"albedo": rmse(alb), "roughness": rmse(rough)},
        "loss_form": "image" if args.image_loss else "fused_l2",
        "peak_autograd_bytes": int(torch.cuda.max_memory_allocated() - mem0),
        "workspace_bytes": dctx.query_workspace(adj), "tuning": tuning,
    }
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
