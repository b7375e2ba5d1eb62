#!/usr/bin/env python
"""Throughput benchmark of the polarized path tracer (primal + cached-suffix-replay adjoint).

One step = one inverse-rendering gradient evaluation of the 50k-triangle displaced
icosphere workload (256x256, 64 spp, depth 8, rough conductor + rough dielectric
pBRDFs, 128^2x3 albedo and 128^2 roughness maps): render_primal (PRB phase 1), the L2
loss adjoint dI = 2 (I - T) / N, render_adjoint (phases 2+3) into both maps.
Metric: primal + adjoint paths per second (each step traces 2 x 4,194,304 paths).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 runs under torchrun: every rank renders its own independent view stream (weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "primal+adjoint paths/sec and gradient MB vs plain launch at 1e-3 grad rel-err"
UNIT = "paths/s"
WORKLOAD = "icosphere50k_256x256_64spp_depth8"

# Algorithmic FP32 work per unit (flops), counted from the operations the method
# performs: a BVH node visit tests two child boxes (12 FMA = 24 flops), a ray/triangle
# test ~30 flops, a ray/sphere test ~20.  Per surface vertex and pass: sampling and the
# light-sample setup 60 (shade stage); the Mueller evaluation and cache store 358
# (rotations 12, Fresnel 60, GGX D*G 40, next-event estimation 150, fold 96); the
# replay 620 (dual-number derivatives of the 262-flop evaluation, ~2x = 524, and the
# adjoint row update a^T W = 96).  The megakernels do the same work in one kernel and trace
# every ray again in the replay; the wavefront's replay reads the cache pass's hits instead.
F_NODE, F_TRI, F_SPH = 24, 30, 20
F_SHADE, F_CACHE, F_REPLAY = 60, 358, 620
F_VERTEX_PRIMAL = F_SHADE + F_CACHE
F_VERTEX_ADJOINT = 2 * F_SHADE + F_CACHE + F_REPLAY

# Algorithmic DRAM bytes of the cache pass (k_wf_finish<MODE, 0>, HBM-bound), per unit:
# per traced ray (a live path of the pass) the list index, bookkeeping, walk and the vertex
# record's ids (4 + 16 + 64 + 16); per surface vertex the rest of the vertex record and the
# visibility (96 + 4), the cache write (124 B of E_v / W_v, + 4 B visibility in the adjoint),
# the walk, bookkeeping and next-list writes (64 + 4 + 4), and the fold's read of the cache
# (124); per finished path the raw Stokes write (48) and, in the adjoint, the image adjoint
# read, the adjoint row write and the replay's start (48 + 48 + 64 + 4 + 4).
B_CACHE_RAY = 100
B_CACHE_VERTEX_PRIMAL, B_CACHE_VERTEX_ADJOINT = 420, 424
B_CACHE_PATH_PRIMAL, B_CACHE_PATH_ADJOINT = 48, 216

# DRAM traffic per launch (bytes) from one ncu capture of this workload: mean of
# dram__bytes_read.sum + dram__bytes_write.sum over the launches of one timed step;
# None for a kernel changed since its capture.
DRAM_BYTES_PER_LAUNCH = {"wf_extend": 269.25e6, "wf_cache": 496.24e6}


# floats per vertex of the wavefront cache: E_v 12, compact W_v 19, the hit 4, visibility 1
WF_CACHE_FLOATS = 36


def wave_paths(job) -> int:
    """Paths per wavefront wave: at most 4,194,304 whole pixels and at most 32 GiB of path
    state (416 B) plus cache (144 B per vertex) per wave, as the library sizes them."""
    per_path = 416 + 4 * WF_CACHE_FLOATS * job.max_depth
    cap = min(1 << 22, (32 << 30) // per_path)
    return min(job.num_paths, max(job.spp, cap // job.spp * job.spp))


def cache_pass_bytes(w: dict, passes: int) -> float:
    """Algorithmic DRAM bytes of the cache pass over the work counted in `w`."""
    if passes == 2:
        return B_CACHE_RAY * w["rays"] + B_CACHE_VERTEX_ADJOINT * w["vertices"] + B_CACHE_PATH_ADJOINT * w["paths"]
    return B_CACHE_RAY * w["rays"] + B_CACHE_VERTEX_PRIMAL * w["vertices"] + B_CACHE_PATH_PRIMAL * w["paths"]


def stage_flops(w: dict, passes: int) -> dict:
    """Algorithmic flops of each stage for one launch of the work counted in `w`."""
    closest = F_NODE * w["nodes"] + F_TRI * w["tri_tests"] + F_SPH * w["sph_tests"]
    shadow = F_NODE * w["shadow_nodes"] + F_TRI * w["shadow_tri_tests"] + F_SPH * w["shadow_sph_tests"]
    V = w["vertices"]
    out = {"wf_extend": closest, "wf_shadow": shadow, "wf_shade": V * F_SHADE, "wf_cache": V * F_CACHE}
    if passes == 2:
        out["wf_replay"] = V * (F_REPLAY + F_SHADE)     # the replay kernels shade their own vertices
        out["adjoint"] = 2 * (closest + shadow) + V * F_VERTEX_ADJOINT
    else:
        out["primal"] = closest + shadow + V * F_VERTEX_PRIMAL
    return out


L2_FLUSH_BYTES = 512 << 20


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time); x itself when world == 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(paths_per_step: int, world: int, steps: int, max_total_ms: float) -> float:
    """Whole-job paths/s: every rank traced paths_per_step paths per step; the job took
    as long as its slowest rank."""
    return paths_per_step * world * steps / (max_total_ms / 1000.0)


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "_source": "fallback"}


# ---------------------------------------------------------------- CPU oracle leg
_W = {}


def _oracle_init(workload_kw):
    import oracle
    from paper_2607_13265_gb300 import scenegen as sg
    oracle.build()
    scene, job = sg.icosphere_scene(**workload_kw)
    _W["o"] = oracle.OracleScene(scene)
    _W["scene"], _W["job"] = scene, job


def _oracle_task(pixels):
    import copy
    import numpy as np
    o, scene, job = _W["o"], _W["scene"], _W["job"]
    pix = np.asarray(pixels, np.int64)
    P = scene.params()
    t0 = time.perf_counter()
    img = o.render(job, P, pixels=pix)
    aj = copy.copy(job)
    aj.pass_id = 1
    o.gradient(aj, P, np.ones_like(img), pixels=pix, mode="replay")
    return time.perf_counter() - t0, 2 * len(pix) * job.spp


def _oracle_tape_task(pixels):
    """Conventional taped AD of the workload's paths on a few pixels: the tape's nodes (one
    per parameter-dependent scalar operation, all kept until the reverse sweep) and the
    vertices they cover."""
    import copy
    import numpy as np
    import oracle
    o, scene, job = _W["o"], _W["scene"], _W["job"]
    pix = np.asarray(pixels, np.int64)
    P = scene.params()
    aj = copy.copy(job)
    aj.pass_id = 1
    img = o.render(aj, P, pixels=pix)
    oracle.stats(reset=True)
    o.gradient(aj, P, np.ones_like(img), pixels=pix, mode="tape")
    st = oracle.stats(reset=True)
    return st["tape_total_nodes"], st["vertices"]


def tape_model(pool, num_pixels: int = 64) -> dict:
    """Tape nodes per path vertex of conventional AD on an evenly strided pixel sample."""
    import numpy as np
    pix = np.linspace(0, 256 * 256 - 1, num_pixels).astype(np.int64)
    res = pool.map(_oracle_tape_task, [pix[i:i + 8].tolist() for i in range(0, len(pix), 8)])
    nodes, verts = sum(r[0] for r in res), sum(r[1] for r in res)
    return {"tape_nodes_per_vertex": nodes / max(verts, 1), "sample": f"{num_pixels} pixels x 64 spp, FP64 oracle tape"}


def oracle_sample(num_pixels: int, procs: int, workload_kw: dict, pool=None):
    """The FP64 oracle (primal + cached-replay adjoint) on an evenly strided pixel
    sample of the workload, one task per 64 pixels over `procs` worker processes."""
    import numpy as np
    npix = 256 * 256
    pix = np.linspace(0, npix - 1, num_pixels).astype(np.int64)
    chunks = [pix[i:i + 64].tolist() for i in range(0, len(pix), 64)]
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_init, initargs=(workload_kw,))
        pool.map(_oracle_task, [chunks[0][:1]] * procs)   # warm every worker
    t0 = time.perf_counter()
    res = pool.map(_oracle_task, chunks)
    wall = time.perf_counter() - t0
    if own:
        pool.close()
        pool.join()
    paths = sum(r[1] for r in res)
    return {"value": paths / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{num_pixels} evenly strided pixels x 64 spp of the {WORKLOAD} workload "
                      f"({paths} primal+adjoint paths, FP64, {wall:.2f} s wall on {procs} processes)",
            "wall_s": wall, "paths": paths}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        if self.proc is not None:
            # the timed region starts once the sampler runs; its first line, taken before the
            # region, is not counted
            import select
            ready, _, _ = select.select([self.proc.stdout], [], [], 10.0)
            if ready:
                self.proc.stdout.readline()
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- native leg
def run_native(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    rank, world, local = _env_rank()
    pool = None
    cpu_procs = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's worker processes are spawned before the first CUDA call
        pool = mp.get_context("spawn").Pool(cpu_procs, initializer=_oracle_init, initargs=({},))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2607_13265_gb300 import api, build, scenegen as sg
    build.build()
    dev = torch.device("cuda", local)
    kw = {}
    if args.width:
        kw["width"] = args.width
    if args.spp:
        kw["spp"] = args.spp
    scene, job = sg.icosphere_scene(**kw)
    job.stream = rank                      # every rank traces its own independent paths
    target_scene, tjob = sg.icosphere_scene(**kw)
    tp = target_scene.params()
    rng = np.random.default_rng(100)
    off, w, h, ch = target_scene.tex_desc[0]
    tp["tex"][off:off + w * h * ch] = rng.uniform(0.2, 0.9, w * h * ch)
    off, w, h, ch = target_scene.tex_desc[1]
    tp["tex"][off:off + w * h * ch] = rng.uniform(0.05, 0.5, w * h * ch)

    dctx = api.Context(local)
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    adj = api.pack_jobs(api.adjoint_jobs([job]))
    P = api.device_params(scene, batch)
    tuning = None
    if args.schedule is not None:
        adj_s = args.schedule if args.adj_schedule is None else args.adj_schedule
        adj_b = args.block if args.adj_block is None else args.adj_block
        dctx.set_launch(args.schedule, args.block, 0, adj_s, adj_b, 0, args.adj_scatter)
    else:
        # the library's autotuner picks schedule and block size for each call (untimed)
        tuning = api.autotune(dctx, gs, adj, P, reps=2)
    tjob.seed = 12345
    target = api.render_primal(dctx, gs, api.pack_jobs([tjob]), api.device_params(scene, batch, tp)).clone()
    N = float(target.numel())
    grads = api.zero_grads(P)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        img = api.render_primal(dctx, gs, batch, P, stream=stream)
        dI = (img - target).mul_(2.0 / N)
        api.render_adjoint(dctx, gs, adj, P, dI, grads, stream=stream)
        return img

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dctx.sync_status()

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    with ClockSampler(local) as clk:                # clocks sampled from here to the end of the region
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        dctx.stage_stats(timing=True, reset=True)  # per-stage CUDA events on the launching stream
        for k in range(K):
            flush.zero_()                               # L2 flush between timed steps (outside the events)
            e0, e1, e2, e3 = ev[k]
            e0.record(stream)
            img = api.render_primal(dctx, gs, batch, P, stream=stream)
            e1.record(stream)
            dI = (img - target).mul_(2.0 / N)
            e2.record(stream)
            api.render_adjoint(dctx, gs, adj, P, dI, grads, stream=stream)
            e3.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    stages = dctx.stage_stats(timing=False, reset=True)
    dctx.sync_status()
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    prim_ms = [e[0].elapsed_time(e[1]) for e in ev]
    adj_ms = [e[2].elapsed_time(e[3]) for e in ev]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    paths_per_step = 2 * job.num_paths
    value = weak_scaling_value(paths_per_step, world, K, total_ms)

    # ---- end to end through the public autograd API with host buffers
    e2e = None
    if rank == 0 or world > 1:
        host_tex = torch.from_numpy(np.asarray(scene.params()["tex"], np.float32)).pin_memory()
        host_grad = torch.empty_like(host_tex).pin_memory()
        host_loss = torch.empty(1, dtype=torch.float32).pin_memory()
        tex_d = P["tex"].clone().requires_grad_(True)
        others = {k: P[k].clone().requires_grad_(True) for k in ("ior", "le", "sheet", "theta")}

        def e2e_step():
            tex_d.data.copy_(host_tex, non_blocking=True)
            tex_d.grad = None
            img = api.PolarizedRender.apply(dctx, gs, batch, adj, tex_d, others["ior"], others["le"],
                                            others["sheet"], others["theta"])
            loss = ((img - target) ** 2).mean()
            loss.backward()
            host_grad.copy_(tex_d.grad, non_blocking=True)
            host_loss.copy_(loss.detach().view(1), non_blocking=True)

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(K):
            flush.zero_()
            a.record(stream)
            e2e_step()
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
        e2e = {"value": paths_per_step * K / (ms / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(host_tex.numel() * 4),
               "d2h_bytes_per_step": int(host_grad.numel() * 4 + 4),
               "api": "PolarizedRender.apply + loss.backward()"}

    # ---- roofline of the dominant kernel (largest share of the timed region's GPU time)
    work = api.count_work(dctx, gs, adj, P)
    pw = api.count_work(dctx, gs, batch, P)
    lc = dctx.get_launch()
    flops = {}
    for name, v in stage_flops(work, 2).items():
        flops[name] = flops.get(name, 0) + v * K
    for name, v in stage_flops(pw, 1).items():
        if name == "primal" or lc[0] == 2:
            flops[name] = flops.get(name, 0) + v * K
    timed = {k: v for k, v in stages.items() if v[0] > 0}
    if "wf_extend" in timed and "wf_shade" not in timed and "wf_shade" in flops:
        # the library shades each cache-pass vertex inside the extend kernel
        flops["wf_extend"] = flops.get("wf_extend", 0) + flops.pop("wf_shade")
    dom = max(timed, key=lambda k: timed[k][1])
    dom_launches, dom_ms = timed[dom]
    adj_avg = sum(adj_ms) / K
    prim_avg = sum(prim_ms) / K
    props = torch.cuda.get_device_properties(dev)
    peaks = load_peaks()
    clocks = clk.summary()
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12        # TFLOP/s at max clock
    fp32_peak_loaded = props.multi_processor_count * 128 * 2 * (clocks["sm_mhz"] or sm_max) * 1e6 / 1e12
    achieved = flops.get(dom, 0) / (dom_ms / 1000.0) / 1e12 if dom_ms > 0 else 0.0
    fp = dctx.adjoint_footprint(job.max_depth)
    cache_bytes = fp["local_bytes_per_thread"] * fp["threads_per_sm"] * fp["sms"]
    stage_report = {k: {"launches": n, "ms_per_step": ms / K,
                        "tflops": (flops[k] / (ms / 1000.0) / 1e12) if k in flops and ms > 0 else None}
                    for k, (n, ms) in timed.items()}
    if "wf_cache" in stage_report and timed["wf_cache"][1] > 0:
        cb = (cache_pass_bytes(work, 2) + (cache_pass_bytes(pw, 1) if lc[0] == 2 else 0)) * K
        stage_report["wf_cache"]["gbs"] = cb / (timed["wf_cache"][1] / 1000.0) / 1e9

    # the dominant kernel's roofline: the cache pass moves records (HBM-bound); traversal and
    # the dual-number replay are bound by FP32 arithmetic issued under divergence
    hbm_peak = float(peaks.get("hbm_gbs") or 6800.0)
    launch_s = dom_ms / max(dom_launches, 1) / 1e3
    traffic = DRAM_BYTES_PER_LAUNCH.get(dom)
    if dom == "wf_cache":
        byt = (cache_pass_bytes(work, 2) + (cache_pass_bytes(pw, 1) if lc[0] == 2 else 0)) * K
        ach = byt / max(dom_launches, 1) / launch_s / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                    "frac": ach / hbm_peak, "traffic": traffic,
                    "bytes_per_launch": byt / max(dom_launches, 1), "launch_ms": launch_s * 1e3,
                    "work_units_adjoint_pass": work,
                    "peak_note": f"{peaks['_source']} HBM copy bandwidth"}
    else:
        roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                    "frac_at_loaded_clock": achieved / fp32_peak_loaded,
                    "traffic": traffic,
                    "hbm": ({"achieved_gbs": traffic / launch_s / 1e9, "peak_gbs": hbm_peak,
                             "frac": traffic / launch_s / 1e9 / hbm_peak,
                             "note": "ncu DRAM bytes per launch (cold caches) / in-bench launch time"}
                            if traffic else None),
                    "flops_per_launch": flops.get(dom, 0) / max(dom_launches, 1),
                    "launch_ms": launch_s * 1e3,
                    "work_units_adjoint_pass": work,
                    "peak_note": f"FP32 pipe: {props.multi_processor_count} SMs x 128 lanes x 2 x {sm_max:.0f} MHz "
                                 f"({peaks['_source']} max clock)"}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded procedural scene, textures and target)",
        "config": {"workload": WORKLOAD if not kw else f"{WORKLOAD} reduced {kw}", "triangles": int(scene.num_triangles), "width": job.width,
                   "height": job.height, "spp": job.spp, "max_depth": job.max_depth,
                   "paths_per_step": paths_per_step, "grads": "albedo 128x128x3 + roughness 128x128",
                   "l2": "flushed between timed steps (512 MiB write)",
                   "schedule": {"primal": [api.SCHEDULE_NAMES[lc[0]], lc[1]], "adjoint": [api.SCHEDULE_NAMES[lc[3]], lc[4]],
                                "adjoint_texel_scatter": ("warp", "lane")[lc[6]],
                                "chosen_by": "autotuner" if tuning else "command line"},
                   "parallelism": f"replicas{world}"},
        "calls_ms": {"render_primal": prim_avg, "render_adjoint": adj_avg},
        "stages": stage_report,
        "roofline": roofline,
        "memory": {"workspace_bytes": dctx.query_workspace(adj),
                   "prb_cache_bytes": (wave_paths(job) * job.max_depth * WF_CACHE_FLOATS * 4 if lc[3] == 2 else cache_bytes),
                   "prb_cache_where": "wavefront workspace" if lc[3] == 2 else "megakernel thread-local memory",
                   "megakernel_local_bytes_per_thread": fp["local_bytes_per_thread"],
                   "megakernel_adjoint_registers": fp["registers"]},
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": int(sum(n for n, _ in timed.values())),
    }
    if pool is not None:
        result["cpu_baseline"] = oracle_sample(args.cpu_pixels, cpu_procs, {}, pool)
        tm = tape_model(pool)
        # conventional AD keeps every path's tape at once: nodes/vertex x vertices of the
        # gradient pass, at 16 B per node (FP32 partials + 32-bit operand indices) and 4 B
        # (one FP32 value: a lower bound for any tape)
        nv = tm["tape_nodes_per_vertex"] * work["vertices"]
        result["memory"]["tape_ad_model"] = {"bytes_16B_per_node": int(16 * nv), "bytes_4B_lower_bound": int(4 * nv),
                                             **tm}
        result["memory"]["prb_cache_vs_tape_ad"] = result["memory"]["prb_cache_bytes"] / max(1.0, 16 * nv)
        pool.close()
        pool.join()
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- reference leg (the oracle)
def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    procs = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_init, initargs=({},))
    pool.map(_oracle_task, [[0]] * procs)
    for _ in range(args.warmup):
        oracle_sample(args.ref_pixels, procs, {}, pool)
    vals, walls, paths = [], 0.0, 0
    for _ in range(args.steps):
        r = oracle_sample(args.ref_pixels, procs, {}, pool)
        walls += r["wall_s"]
        paths += r["paths"]
    pool.close()
    pool.join()
    value = paths / walls
    sample = (f"{args.ref_pixels} evenly strided pixels x 64 spp of the {WORKLOAD} workload per step "
              f"(FP64 oracle: primal + cached-replay adjoint)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * walls / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded procedural scene)", "config": {"workload": WORKLOAD, "parallelism": f"cpu{procs}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--schedule", type=int, default=None, help="0 grid, 1 persistent (default: library default)")
    ap.add_argument("--block", type=int, default=128)
    ap.add_argument("--adj-schedule", type=int, default=None, help="adjoint schedule (default: same as --schedule)")
    ap.add_argument("--adj-block", type=int, default=None)
    ap.add_argument("--adj-scatter", type=int, default=0, choices=[0, 1],
                    help="with --schedule: texel gradients per warp group (0) or per lane (1)")
    ap.add_argument("--cpu-pixels", type=int, default=16384)
    ap.add_argument("--ref-pixels", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--width", type=int, default=None, help="smaller image (profiling captures only)")
    ap.add_argument("--spp", type=int, default=None, help="fewer samples per pixel (profiling captures only)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
