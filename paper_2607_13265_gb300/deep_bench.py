"""Deep-path benchmark: time and memory of the gradient pass versus path depth.

Workload (scenegen.deep_stack_scene): a closed diffuse room with a rough-conductor mesh and
a stack of 85 linear polarizers twisting from 0 to 90 deg, 1280x720, 1 spp, polarizer
camera filter; every path runs to max_depth, and a path through the stack spends 85
vertices in it.  For each max_depth and each schedule the module times render_primal and
render_adjoint (cached suffix replay) with CUDA events on the launching stream, after a
warm-up call, and reports the memory the adjoint holds for its cache (for the fully cached
replay and, with --hybrid k.., for the hybrid cached replay of Sec. 4.4 with checkpoints
every k vertices; with --pprb, for the basic polarized PRB baseline, which keeps no cache):
  * megakernel schedules: the per-thread local cache (bytes per thread, from the compiled
    kernel) times the threads resident on the GPU -- independent of the image size;
  * wavefront and sweep schedules: the library workspace (path state + per-vertex cache of
    one wave, waves capped at 32 GiB; with the hybrid, each vertex's hit and the checkpoint
    data instead of the cache; the sweep's megakernel also holds the thread-local cache of
    its resident threads).  --hybrid runs on every schedule given with --hybrid-schedules.
The loss is a seeded linear functional of the image.  Prints one JSON line per
(schedule, depth) and a final summary line.

  python -m paper_2607_13265_gb300.deep_bench [--depths 4 8 16 32 64 128] [--reps 3] [--hybrid 4 8 16]
      [--pprb 0.01]
"""
from __future__ import annotations

import argparse
import copy
import json

import numpy as np

SCHEDULE_IDS = {"grid": 0, "persistent": 1, "wavefront": 2, "sweep": 3}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--depths", type=int, nargs="+", default=[4, 8, 16, 32, 64, 128])
    ap.add_argument("--schedules", nargs="+", default=["grid", "wavefront"], choices=list(SCHEDULE_IDS))
    ap.add_argument("--block", type=int, default=128)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--width", type=int, default=1280)
    ap.add_argument("--height", type=int, default=720)
    ap.add_argument("--sheets", type=int, default=85)
    ap.add_argument("--hybrid", type=int, nargs="*", default=[], help="checkpoint intervals k of hybrid replay runs")
    ap.add_argument("--hybrid-schedules", nargs="+", default=["grid"], choices=list(SCHEDULE_IDS))
    ap.add_argument("--gamma", type=float, default=0.0)
    ap.add_argument("--eps", type=float, default=float("inf"))
    ap.add_argument("--pprb", type=float, default=None,
                    help="also time the basic polarized PRB baseline with this noise deviation")
    args = ap.parse_args(argv)

    import torch
    from . import api, build, scenegen as sg
    build.build()
    scene, job0 = sg.deep_stack_scene(num_sheets=args.sheets, width=args.width, height=args.height, spp=1,
                                      depth=max(args.depths))
    dctx = api.Context(0)
    gs = api.GpuScene(dctx, scene)
    stream = torch.cuda.Stream()
    rows = []
    runs = [(s_, 1, "cached") for s_ in args.schedules] + [(s_, k, "cached") for s_ in args.hybrid_schedules
                                                                 for k in args.hybrid]
    if args.pprb is not None:
        runs.append(("grid", 1, "pprb"))
    for sched, kint, method in runs:
        dctx.set_replay(kint, args.gamma, args.eps, method=method, sigma=args.pprb or 0.0)
        label = "grid/pprb" if method == "pprb" else sched if kint == 1 else f"{sched}/hybrid-k{kint}"
        for d in args.depths:
            job = copy.copy(job0)
            job.max_depth = d
            batch = api.pack_jobs([job])
            adj = api.pack_jobs(api.adjoint_jobs([job]))
            P = api.device_params(scene, batch)
            dctx.set_launch(SCHEDULE_IDS[sched], args.block, 0)
            dI = torch.as_tensor(np.random.default_rng(3).normal(size=batch.image_floats), dtype=torch.float32,
                                 device="cuda")
            grads = api.zero_grads(P)
            img = torch.empty(batch.image_floats, dtype=torch.float32, device="cuda")
            free0 = torch.cuda.mem_get_info()[0]
            with torch.cuda.stream(stream):
                api.render_primal(dctx, gs, batch, P, image=img, stream=stream)
                api.render_adjoint(dctx, gs, adj, P, dI, grads, stream=stream)
            stream.synchronize()
            dctx.sync_status(stream)
            grown = free0 - torch.cuda.mem_get_info()[0]
            tp, ta = [], []
            for _ in range(args.reps):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                with torch.cuda.stream(stream):
                    e[0].record(stream)
                    api.render_primal(dctx, gs, batch, P, image=img, stream=stream)
                    e[1].record(stream)
                    api.render_adjoint(dctx, gs, adj, P, dI, grads, stream=stream)
                    e[2].record(stream)
                e[2].synchronize()
                tp.append(e[0].elapsed_time(e[1]))
                ta.append(e[1].elapsed_time(e[2]))
            dctx.sync_status(stream)
            work = api.count_work(dctx, gs, adj, P)
            fp = dctx.adjoint_footprint(d)
            ws = dctx.query_workspace(adj)
            mega_cache = fp["local_bytes_per_thread"] * fp["threads_per_sm"] * fp["sms"]
            row = {"schedule": label, "depth": d, "paths": job.num_paths,
                   "vertices_per_path": work["vertices"] / job.num_paths,
                   "primal_ms": float(np.median(tp)), "adjoint_ms": float(np.median(ta)),
                   "adjoint_vertices_per_s": work["vertices"] / (float(np.median(ta)) / 1e3),
                   "cache_bytes": int(ws if sched in ("wavefront", "sweep") else mega_cache),
                   "replay": {"method": method, "checkpoint_interval": kint, "gamma": args.gamma, "eps": args.eps,
                              "sigma": args.pprb if method == "pprb" else None},
                   "workspace_bytes": int(ws), "local_bytes_per_thread": int(fp["local_bytes_per_thread"]),
                   "resident_threads": int(fp["threads_per_sm"] * fp["sms"]),
                   "device_bytes_grown_first_call": int(grown),
                   "grad_norm": {k: float(v.norm()) for k, v in grads.items() if v.numel()}}
            rows.append(row)
            print(json.dumps(row), flush=True)
    dctx.set_replay(1)
    print(json.dumps({"workload": f"deep_stack{args.sheets}_{args.width}x{args.height}_1spp",
                      "summary": [(r["schedule"], r["depth"], round(r["primal_ms"], 2), round(r["adjoint_ms"], 2),
                                   r["cache_bytes"]) for r in rows]}))
    return rows


if __name__ == "__main__":
    main()
