"""Sweep of hybrid cached replay's thresholds (Sec. 4.4, Eq. hybrid_decision): gradient
error against the exact gradient, adjoint time and cache memory, for checkpoint intervals k
and thresholds gamma (depolarization index below which a block is replayed as scalar PRB)
and eps (|det| above which a block's throughput is inverted); the rest is recomputed.

Workloads: 'deep', the deep-path scene (scenegen.deep_stack_scene: closed diffuse room, a
rough conductor mesh and a stack of 85 twisting linear polarizers), 1280x720, 1 spp, max
depth 64 -- its blocks are depolarizing (diffuse: depolarization index 0, determinant 0) or
hold an ideal polarizer (index 1, determinant 0), so the scalar route is exact where it is
taken and no block is inverted; 'rocks', the rough-dielectric rocks (scenegen.rocks_scene,
GGX specular + depolarizing lobe, index of refraction 1.3-1.7: partially polarizing blocks
with nonzero determinants) behind a quarter-wave plate and a polarizer, max depth 16, where
the thresholds do choose approximate routes.  A seeded linear loss on the image.
Reference: the fully cached replay (k = 1), which equals the FP64 oracle's gradient within
the parity tolerance.  For each (k, gamma, eps): the relative L2 error of every gradient
group, the adjoint time (CUDA events, median of `reps`) and the memory of the replay: on
the grid schedule the per-thread local cache of the megakernel times the resident threads,
on the wavefront the library workspace.  Prints one JSON line per configuration and a
summary line.

  python -m paper_2607_13265_gb300.hybrid_sweep [--scene deep|rocks] [--schedule grid|wavefront]
      [--depth 64] [--ks 4 8 16] [--gammas ...] [--epss ...]
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--scene", choices=["deep", "rocks"], default="deep")
    ap.add_argument("--depth", type=int, default=None, help="max depth (default: 64 deep, 16 rocks)")
    ap.add_argument("--spp", type=int, default=None, help="samples per pixel (default: 1 deep, 8 rocks)")
    ap.add_argument("--ks", type=int, nargs="+", default=[4, 8, 16])
    ap.add_argument("--gammas", type=float, nargs="+", default=[0.0, 0.05, 0.2, 0.5, 1.0])
    ap.add_argument("--epss", type=float, nargs="+", default=[float("inf"), 1e-1, 1e-3, 1e-6])
    ap.add_argument("--width", type=int, default=None, help="default: 1280 deep, 256 rocks")
    ap.add_argument("--height", type=int, default=None, help="default: 720 deep, 256 rocks")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--schedule", choices=["grid", "wavefront"], default="grid")
    args = ap.parse_args(argv)

    import torch
    from . import api, build, scenegen as sg
    build.build()
    deep = args.scene == "deep"
    W_, H_ = args.width or (1280 if deep else 256), args.height or (720 if deep else 256)
    depth, spp = args.depth or (64 if deep else 16), args.spp or (1 if deep else 8)
    if deep:
        scene, job = sg.deep_stack_scene(width=W_, height=H_, spp=spp, depth=depth)
    else:
        scene, job = sg.rocks_scene(width=W_, spp=spp, depth=depth)
        job.height = H_
    dctx = api.Context(0)
    gs = api.GpuScene(dctx, scene)
    adj = api.pack_jobs(api.adjoint_jobs([job]))
    P = api.device_params(scene, adj)
    dI = torch.as_tensor(np.random.default_rng(3).normal(size=adj.image_floats), dtype=torch.float32, device="cuda")
    wave = args.schedule == "wavefront"
    dctx.set_launch(2 if wave else 0, 128, 0)

    def run(k, gamma, eps):
        dctx.set_replay(k, gamma, eps)
        g = api.render_adjoint(dctx, gs, adj, P, dI)          # warm-up (and the result)
        dctx.sync_status()
        times = []
        for _ in range(args.reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            api.render_adjoint(dctx, gs, adj, P, dI, api.zero_grads(P))
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
        dctx.sync_status()
        fp = dctx.adjoint_footprint(job.max_depth)
        cache = dctx.query_workspace(adj) if wave else fp["local_bytes_per_thread"] * fp["threads_per_sm"] * fp["sms"]
        return {n: v.double().cpu().numpy() for n, v in g.items()}, float(np.median(times)), int(cache)

    ref, t_ref, cache_ref = run(1, 0.0, float("inf"))
    groups = {}
    for t, (off, w, h, ch) in enumerate(scene.tex_desc):
        if scene.tex_differentiable[t]:
            groups[f"tex{t}"] = (lambda o, n: lambda g: g["tex"][o:o + n])(int(off), int(w * h * ch))
    for name in ("ior", "sheet", "le", "theta"):
        groups[name] = (lambda k_: lambda g: g[k_])(name)

    def errors(g):
        out = {}
        for n, f in groups.items():
            o = f(ref)
            out[n] = float(np.linalg.norm(f(g) - o) / np.linalg.norm(o)) if np.linalg.norm(o) > 0 else None
        return out

    rows = [{"k": 1, "gamma": 0.0, "eps": "inf", "adjoint_ms": t_ref, "cache_bytes": cache_ref, "errors": errors(ref)}]
    print(json.dumps(rows[0]), flush=True)
    for k in args.ks:
        for gamma in args.gammas:
            for eps in args.epss:
                g, t, cache = run(k, gamma, eps)
                row = {"k": k, "gamma": gamma, "eps": eps if np.isfinite(eps) else "inf", "adjoint_ms": t,
                       "cache_bytes": cache, "errors": errors(g)}
                rows.append(row)
                print(json.dumps(row), flush=True)
    dctx.set_replay(1)
    print(json.dumps({"workload": (f"deep_stack85_{W_}x{H_}_{spp}spp_depth{depth}" if deep
                                   else f"rocks100k_{W_}x{H_}_{spp}spp_depth{depth}"), "schedule": args.schedule,
                      "reference": "fully cached replay (k = 1)",
                      "summary": [(r["k"], r["gamma"], r["eps"], round(r["adjoint_ms"], 1), r["cache_bytes"],
                                   {n: (round(v, 5) if v is not None else None) for n, v in r["errors"].items()})
                                  for r in rows]}))
    return rows


if __name__ == "__main__":
    main()
