"""Batched versus plain gradient evaluation of many polarizer angles and views.

Workload: the Cornell-box scene seen from 8 cameras orbiting +-20 deg in yaw with square
image sizes 128..512 (945,372 pixels in all), each behind a linear polarizer at 64 angles
in [0, 180) deg; 16 spp, depth 8; L2 loss to a seeded target (perturbed albedo).

* batched: all views and angles in ONE render_primal and ONE render_adjoint call (the
  views in one launch; the angles folded exactly, since the filter does not change the
  paths), the whole gradient step captured in a CUDA graph and replayed; p50/p99 per batch.
* plain: one call per (view, angle), i.e. 512 render_primal + 512 render_adjoint calls,
  each tracing the view's paths again.

* batched, fused L2: the same batch with the loss folded into the camera filter
  (PolarizedL2 / dppt_loss_l2 + dppt_render_adjoint_l2): only the raw image (12 floats per
  pixel) is kept instead of one image per angle, captured in a CUDA graph as well.

All forms run through their autograd Functions for the memory comparison (peak device
memory of forward + backward, plus the library's workspace).  Prints one JSON line.

  python -m paper_2607_13265_gb300.batch_bench [--replays 50] [--angles 64] [--views 8]
"""
from __future__ import annotations

import argparse
import copy
import json

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--replays", type=int, default=50)
    ap.add_argument("--angles", type=int, default=64)
    ap.add_argument("--views", type=int, default=8)
    ap.add_argument("--spp", type=int, default=16)
    ap.add_argument("--depth", type=int, default=8)
    ap.add_argument("--scale", type=float, default=1.0, help="image sides scaled by this factor (tests)")
    ap.add_argument("--no-tune", action="store_true")
    args = ap.parse_args(argv)

    import torch
    from . import api, build, scenegen as sg
    build.build()
    sizes = tuple(max(8, int(round(s * args.scale))) for s in (128, 183, 238, 293, 347, 402, 457, 512))
    scene, jobs = sg.cornell_views(args.views, args.angles, args.spp, args.depth, sizes)
    dctx = api.Context(0)
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs(jobs)
    adj = api.pack_jobs(api.adjoint_jobs(jobs))
    P = api.device_params(scene, batch)
    tuning = None if args.no_tune else api.autotune(dctx, gs, adj, P, reps=1)

    # seeded target: the albedo of the diffuse sphere and of the walls perturbed
    tp = scene.params()
    rng = np.random.default_rng(21)
    tp["tex"] = np.clip(tp["tex"] + rng.uniform(-0.15, 0.15, tp["tex"].shape), 0.05, 0.95)
    tp["theta"] = batch.theta
    tjobs = [copy.copy(j) for j in jobs]
    for j in tjobs:
        j.seed = 777
    target = api.render_primal(dctx, gs, api.pack_jobs(tjobs), api.device_params(scene, batch, tp)).clone()
    N = float(target.numel())
    grads = api.zero_grads(P)
    stream = torch.cuda.Stream()

    def step():
        img = api.render_primal(dctx, gs, batch, P, image=img_buf, stream=stream)
        torch.sub(img, target, out=dI_buf)
        dI_buf.mul_(2.0 / N)
        for g in grads.values():
            g.zero_()
        api.render_adjoint(dctx, gs, adj, P, dI_buf, grads, stream=stream)

    img_buf = torch.empty_like(target)
    dI_buf = torch.empty_like(target)
    with torch.cuda.stream(stream):
        for _ in range(2):
            step()          # warm-up: the library sizes its workspace here, before capture
    stream.synchronize()
    eager = []
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        with torch.cuda.stream(stream):
            step()
        b.record(stream)
        b.synchronize()
        eager.append(a.elapsed_time(b))
    grads_eager = {k: v.clone() for k, v in grads.items()}

    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step()
    lat = []
    for _ in range(args.replays):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):      # a graph replays on the current stream
            a.record(stream)
            graph.replay()
            b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
    dctx.sync_status(stream)
    graph_vs_eager = max(float((grads[k] - grads_eager[k]).abs().max() / (grads_eager[k].abs().max() + 1e-30))
                         for k in ("tex", "theta"))

    # the same step with the L2 loss fused into the camera filter (12 floats per pixel kept)
    rb = api.raw_batch(batch)
    raw_buf = torch.empty(rb.image_floats, dtype=torch.float32, device="cuda")
    loss_buf = torch.empty((), dtype=torch.float64, device="cuda")
    grads_f = api.zero_grads(P)

    def step_fused():
        api.render_primal(dctx, gs, rb, P, image=raw_buf, stream=stream)
        api.loss_l2(dctx, gs, batch, P, raw_buf, rb.offsets, target, 1.0 / N, loss=loss_buf, stream=stream)
        for g in grads_f.values():
            g.zero_()
        api.render_adjoint_l2(dctx, gs, adj, P, raw_buf, rb.offsets, target, 1.0 / N, grads_f, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(2):
            step_fused()
    stream.synchronize()
    fused_vs_image = max(float((grads_f[k] - grads_eager[k]).abs().max() / (grads_eager[k].abs().max() + 1e-30))
                         for k in ("tex", "theta"))
    graph_f = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_f, stream=stream):
        step_fused()
    lat_f = []
    for _ in range(args.replays):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            graph_f.replay()
            b.record(stream)
        b.synchronize()
        lat_f.append(a.elapsed_time(b))
    dctx.sync_status(stream)

    traced = sum(2 * j.num_paths for j in jobs)                       # primal + adjoint paths traced
    effective = sum(2 * j.num_paths * j.num_angles for j in jobs)     # (view, angle) path samples produced
    p50, p99 = float(np.percentile(lat, 50)), float(np.percentile(lat, 99))

    # per-view gradients: dL/dtheta for every (view, angle)
    th = grads["theta"].cpu().numpy()
    per_view = []
    for j, off in zip(jobs, np.cumsum([0] + [k.num_angles for k in jobs])[:-1]):
        g = th[off:off + j.num_angles]
        per_view.append({"size": j.width, "dtheta_l2": float(np.linalg.norm(g)),
                         "dtheta_at_0deg": float(g[0]), "dtheta_at_90deg": float(g[len(g) // 2])})

    # plain form: one call per (view, angle)
    plain_jobs, plain_adj = [], []
    for j in jobs:
        for t in j.thetas:
            k = copy.copy(j)
            k.thetas = [t]
            plain_jobs.append(k)
    plain_batches = [api.pack_jobs([k]) for k in plain_jobs]
    plain_adj = [api.pack_jobs(api.adjoint_jobs([k])) for k in plain_jobs]
    views = api.image_views(batch, target)
    plain_targets = []
    for vi, j in enumerate(jobs):
        for a in range(j.num_angles):
            plain_targets.append(views[vi][a].reshape(-1))
    plain_params = []
    for k, pb in zip(plain_jobs, plain_batches):
        q = dict(P)
        q["theta"] = torch.tensor([k.thetas[0]], dtype=torch.float32, device="cuda")
        plain_params.append(q)
    pg = api.zero_grads(P)
    torch.cuda.synchronize()

    def plain_all():
        for pb, pa, q, t in zip(plain_batches, plain_adj, plain_params, plain_targets):
            img = api.render_primal(dctx, gs, pb, q, stream=stream)
            d = (img - t).mul_(2.0 / N)
            gq = {"tex": pg["tex"], "ior": pg["ior"], "le": pg["le"], "sheet": pg["sheet"],
                  "theta": torch.zeros(1, device="cuda")}
            api.render_adjoint(dctx, gs, pa, q, d, gq, stream=stream)

    with torch.cuda.stream(stream):
        plain_all()                      # warm-up
    stream.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    with torch.cuda.stream(stream):
        plain_all()
    b.record(stream)
    b.synchronize()
    plain_ms = a.elapsed_time(b)
    plain_traced = sum(2 * k.num_paths for k in plain_jobs)

    # gradient memory of the two autograd forms (peak device memory of forward + backward)
    def peak(fn):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        fn()
        torch.cuda.synchronize()
        return torch.cuda.max_memory_allocated() - base

    leaf = {k: v.clone().requires_grad_(True) for k, v in P.items()}

    def batched_autograd():
        img = api.PolarizedRender.apply(dctx, gs, batch, adj, leaf["tex"], leaf["ior"], leaf["le"], leaf["sheet"],
                                        leaf["theta"])
        api.ImageL2.apply(img, target).backward()

    def plain_autograd():
        loss = 0.0
        for pb, pa, q, t in zip(plain_batches, plain_adj, plain_params, plain_targets):
            thq = q["theta"].clone().requires_grad_(True)
            img = api.PolarizedRender.apply(dctx, gs, pb, pa, leaf["tex"], leaf["ior"], leaf["le"], leaf["sheet"], thq)
            loss = loss + api.ImageL2.apply(img, t) * (img.numel() / N)
        loss.backward()

    def fused_autograd():
        loss = api.PolarizedL2.apply(dctx, gs, batch, adj, target, leaf["tex"], leaf["ior"], leaf["le"],
                                     leaf["sheet"], leaf["theta"])
        loss.backward()

    mem_batched = peak(batched_autograd)
    ws_batched = dctx.query_workspace(adj)
    mem_fused = peak(fused_autograd)
    mem_plain = peak(plain_autograd)
    ws_plain = max(dctx.query_workspace(pa) for pa in plain_adj[:: max(1, args.angles)])

    lc = dctx.get_launch()
    out = {
        "workload": f"cornell_views{args.views}x{args.angles}angles_{args.spp}spp_depth{args.depth}",
        "pixels": int(sum(j.num_pixels for j in jobs)), "sizes": list(sizes[:args.views]),
        "schedule": {"primal": [api.SCHEDULE_NAMES[lc[0]], lc[1]], "adjoint": [api.SCHEDULE_NAMES[lc[3]], lc[4]],
                     "chosen_by": "autotuner" if tuning else "default"},
        "batched": {"graph_p50_ms": p50, "graph_p99_ms": p99, "eager_ms": float(np.median(eager)),
                    "traced_paths_per_s": traced / (p50 / 1000.0),
                    "effective_paths_per_s": effective / (p50 / 1000.0),
                    "graph_vs_eager_grad_rel": graph_vs_eager,
                    "peak_autograd_bytes": int(mem_batched), "workspace_bytes": int(ws_batched)},
        "batched_fused_l2": {"graph_p50_ms": float(np.percentile(lat_f, 50)),
                             "graph_p99_ms": float(np.percentile(lat_f, 99)),
                             "traced_paths_per_s": traced / (float(np.percentile(lat_f, 50)) / 1000.0),
                             "effective_paths_per_s": effective / (float(np.percentile(lat_f, 50)) / 1000.0),
                             "grad_rel_vs_image_form": fused_vs_image,
                             "peak_autograd_bytes": int(mem_fused)},
        "plain": {"calls": 2 * len(plain_jobs), "ms": plain_ms, "traced_paths_per_s": plain_traced / (plain_ms / 1000.0),
                  "effective_paths_per_s": effective / (plain_ms / 1000.0),
                  "peak_autograd_bytes": int(mem_plain), "workspace_bytes": int(ws_plain)},
        "speedup_effective": plain_ms / p50,
        "gradient_memory_vs_plain": {"batched_image_form": mem_batched / max(1, mem_plain),
                                     "batched_fused_l2": mem_fused / max(1, mem_plain)},
        "per_view_gradients": per_view,
        "tuning": tuning,
    }
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
