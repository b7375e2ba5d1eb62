#!/usr/bin/env python
"""Throughput benchmark of the polarized path tracer (primal + cached-suffix-replay adjoint).

Headline workload (the batched views x angles gradient): the Cornell-box scene (12
triangles + 2 spheres: diffuse walls, a diffuse and a glass sphere, a quad light) seen by 8
cameras orbiting +-20 deg with square images of 128, 183, 238, 293, 347, 402, 457 and 512
pixels (945,372 pixels), each behind a linear polarizer at 64 angles in [0, 180) deg; 16
spp, depth 8; L2 loss to a seeded target (perturbed albedo, other random numbers).

* One step = one gradient evaluation of the whole batch in its batched autograd form
  (PolarizedL2: render_primal of the raw image of all views in one launch, the loss
  folded into the camera filter, render_adjoint_l2 of all views in one call), captured
  once in a CUDA graph and replayed; the timed region is K replays.
* Metric: primal + adjoint paths per second, counting every (view, angle, pixel, sample)
  path of the primal and of the adjoint -- the paths the plain form traces one call at a
  time (2 x 968,318,976 per step); the batched form traces each view's paths once
  (2 x 15,125,952) and folds the angles exactly.  The same line reports, measured in the
  same run: the plain form (512 render_primal + 512 render_adjoint calls, one per view and
  angle), the traced-path rate of both forms, and the gradient memory (peak device memory
  of forward + backward through torch.autograd) of the batched and the plain form.
* "icosphere": the 50k-triangle displaced icosphere (256x256, 64 spp, depth 8, rough
  conductor + rough dielectric, 128^2x3 albedo and 128^2 roughness maps) as one eager
  gradient step per iteration, with its stage times and the roofline of its dominant kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 runs under torchrun: every rank renders its own independent paths (weak scaling,
no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import copy
import json
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
VIEW_SIZES = (128, 183, 238, 293, 347, 402, 457, 512)
NUM_VIEWS, NUM_ANGLES, VIEW_SPP, VIEW_DEPTH = 8, 64, 16, 8
WORKLOAD = f"cornell_views{NUM_VIEWS}x{NUM_ANGLES}angles_{VIEW_SPP}spp_depth{VIEW_DEPTH}"
ICO_WORKLOAD = "icosphere50k_256x256_64spp_depth8"

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

# DRAM traffic per launch (bytes; dram__bytes_read.sum + dram__bytes_write.sum, cold caches)
# keyed by (workload, stage), for the stages the benchmark's launch shapes run: captured on the
# views workload with every image side halved (3,779,744 paths per pass, one wave) and scaled
# by the paths a full-size launch processes: the primal megakernel 466 B per path (one launch
# of 15,125,952 paths per step), the forward sweep 2,203 B per path (four waves, 3,781,488
# paths per launch on average).  Absent for a kernel changed since its capture.
DRAM_BYTES_PER_LAUNCH = {
    ("cornell_views8x64angles_16spp_depth8", "primal"): 7.052e9,
    ("cornell_views8x64angles_16spp_depth8", "wf_sweep"): 8.329e9,
}

# floats per vertex of the wavefront cache: E_v 12, compact W_v 19, visibility 1, the hit 4
WF_CACHE_FLOATS = 36
# bytes per vertex the sweep schedule keeps for the replay: the suffix 48, the hit 16 and the
# visibility word 4 (besides its megakernel's thread-local arrays)
SWEEP_RECORD_BYTES = 68


def wave_paths(jobs) -> int:
    """Path slots of a wavefront wave, as the library sizes them: all the jobs' paths when
    they fit, else 4,194,304 or fewer when a wave's path state (432 B) plus cache (144 B per
    vertex) would pass 32 GiB; several jobs share a wave."""
    per_path = 432 + 4 * WF_CACHE_FLOATS * max(j.max_depth for j in jobs)
    cap = min(1 << 22, (32 << 30) // per_path)
    return max(max(j.spp for j in jobs), min(sum(j.num_paths for j in jobs), cap))


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
        # the sweep schedule's forward sweep: one megakernel for the adjoint's tracing,
        # shading, evaluation and fold
        out["wf_sweep"] = closest + shadow + V * F_VERTEX_PRIMAL
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


def views_workload(scale: float = 1.0):
    """The views x angles batch (scale < 1 shrinks the image sides, for tests only)."""
    from paper_2607_13265_gb300 import scenegen as sg
    sizes = tuple(max(8, int(round(s * scale))) for s in VIEW_SIZES)
    return sg.cornell_views(NUM_VIEWS, NUM_ANGLES, VIEW_SPP, VIEW_DEPTH, sizes)


def path_counts(jobs) -> tuple[int, int]:
    """(paths counted by the metric, paths traced by the batched form) per gradient step:
    primal + adjoint, the former once per polarizer angle."""
    return (sum(2 * j.num_paths * j.num_angles for j in jobs), sum(2 * j.num_paths for j in jobs))


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


def _oracle_init(scale: float = 1.0):
    import oracle
    oracle.build()
    scene, jobs = views_workload(scale)
    _W["o"] = oracle.OracleScene(scene)
    _W["scene"], _W["jobs"] = scene, jobs


def _oracle_task(item):
    """Primal + cached-replay adjoint of the oracle on some pixels of one view, all angles."""
    import numpy as np
    view, pixels = item
    o, scene, job = _W["o"], _W["scene"], _W["jobs"][view]
    pix = np.asarray(pixels, np.int64)
    P = scene.params()
    t0 = time.perf_counter()
    img = o.render(job, P, pixels=pix)
    aj = copy.copy(job)
    aj.pass_id = 1
    o.gradient(aj, P, np.ones_like(img), pixels=pix, mode="replay")
    return time.perf_counter() - t0, 2 * len(pix) * job.spp * job.num_angles, 2 * len(pix) * job.spp


def _sample_items(num_pixels: int, scale: float = 1.0):
    """num_pixels pixels spread evenly over the views (evenly strided in each), as tasks of
    at most 32 pixels."""
    import numpy as np
    _, jobs = views_workload(scale)
    per = max(1, num_pixels // len(jobs))
    items = []
    for v, j in enumerate(jobs):
        pix = np.linspace(0, j.num_pixels - 1, min(per, j.num_pixels)).astype(np.int64)
        items += [(v, pix[i:i + 32].tolist()) for i in range(0, len(pix), 32)]
    return items


def oracle_sample(num_pixels: int, procs: int, pool=None, scale: float = 1.0):
    """The FP64 oracle (primal + cached-replay adjoint, all 64 angles) on an evenly strided
    pixel sample of the views x angles workload over `procs` worker processes."""
    items = _sample_items(num_pixels, scale)
    own = pool is None
    if own:
        pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_init, initargs=(scale,))
        pool.map(_oracle_task, [(0, [0])] * procs)    # warm every worker
    t0 = time.perf_counter()
    res = pool.map(_oracle_task, items)
    wall = time.perf_counter() - t0
    if own:
        pool.close()
        pool.join()
    paths = sum(r[1] for r in res)
    traced = sum(r[2] for r in res)
    npix = sum(len(p) for _, p in items)
    return {"value": paths / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{npix} evenly strided pixels over the 8 views of the {WORKLOAD} workload, 16 spp, "
                      f"all 64 angles ({traced} primal+adjoint paths traced, {paths} counted as the metric counts "
                      f"them; FP64, {wall:.2f} s wall on {procs} processes)",
            "traced_paths_per_s": traced / wall, "wall_s": wall, "paths": paths}


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


# ---------------------------------------------------------------- roofline
def roofline_of(stages: dict, flops: dict, cache_bytes: float, props, peaks: dict, clocks: dict,
                traffic_key: str, work: dict) -> dict:
    """Roofline of the stage with the most GPU time in `stages` ({stage: (launches, ms)}):
    the cache pass against HBM (records and cache move through DRAM), every other stage
    against the FP32 pipe (traversal and dual-number arithmetic under divergence)."""
    timed = {k: v for k, v in stages.items() if v[0] > 0 and v[1] > 0}
    dom = max(timed, key=lambda k: timed[k][1])
    launches, ms = timed[dom]
    launch_s = ms / launches / 1e3
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    fp32_loaded = props.multi_processor_count * 128 * 2 * (clocks.get("sm_mhz") or sm_max) * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs") or 6800.0)
    traffic = DRAM_BYTES_PER_LAUNCH.get((traffic_key, dom))
    if dom == "wf_cache":
        ach = cache_bytes / launches / launch_s / 1e9
        return {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic, "bytes_per_launch": cache_bytes / launches,
                "launch_ms": launch_s * 1e3, "launches": launches, "work_units_adjoint_pass": work,
                "peak_note": f"{peaks['_source']} HBM copy bandwidth"}
    ach = flops.get(dom, 0) / launches / launch_s / 1e12
    return {"bound": "alu", "kernel": dom, "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": ach / fp32_peak, "frac_at_loaded_clock": ach / fp32_loaded, "traffic": traffic,
            "hbm": ({"achieved_gbs": traffic / launch_s / 1e9, "peak_gbs": hbm_peak,
                     "frac": traffic / launch_s / 1e9 / hbm_peak,
                     "note": "ncu DRAM bytes per launch (cold caches) / in-bench launch time"} if traffic else None),
            "flops_per_launch": flops.get(dom, 0) / launches, "launch_ms": launch_s * 1e3, "launches": launches,
            "work_units_adjoint_pass": work,
            "peak_note": f"FP32 pipe: {props.multi_processor_count} SMs x 128 lanes x 2 x {sm_max:.0f} MHz "
                         f"({peaks['_source']} max clock)"}


def workload_flops(work: dict, pwork: dict, launch: tuple, steps: int) -> tuple[dict, float]:
    """Algorithmic flops per stage and cache-pass bytes of `steps` gradient steps (primal
    work `pwork`, adjoint work `work`) under the launch shapes `launch`."""
    flops = {}
    for name, v in stage_flops(work, 2).items():
        flops[name] = flops.get(name, 0) + v * steps
    for name, v in stage_flops(pwork, 1).items():
        if name == "primal" or launch[0] == 2:
            flops[name] = flops.get(name, 0) + v * steps
    # the library shades each cache-pass vertex inside the extend kernel
    flops["wf_extend"] = flops.get("wf_extend", 0) + flops.pop("wf_shade", 0)
    cb = (cache_pass_bytes(work, 2) + (cache_pass_bytes(pwork, 1) if launch[0] == 2 else 0)) * steps
    return flops, cb


def stage_report(stages: dict, flops: dict, cache_bytes: float, steps: int) -> dict:
    out = {}
    for k, (n, ms) in stages.items():
        if n == 0:
            continue
        r = {"launches_per_step": n / steps, "ms_per_step": ms / steps,
             "tflops": (flops[k] / (ms / 1000.0) / 1e12) if k in flops and ms > 0 else None}
        if k == "wf_cache" and ms > 0:
            r["gbs"] = cache_bytes / (ms / 1000.0) / 1e9
        out[k] = r
    return out


# ---------------------------------------------------------------- native leg
def run_views(args, api, dctx, rank, world, dev, clk_index, peaks):
    """The headline: batched views x angles gradient step in a CUDA graph, the plain form,
    gradient memory of both, end to end through PolarizedL2 with host buffers."""
    import numpy as np
    import torch
    scene, jobs = views_workload(args.scale)
    for j in jobs:
        j.stream += 1000 * rank                  # every rank traces its own independent paths
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs(jobs)
    adj = api.pack_jobs(api.adjoint_jobs(jobs))
    rb = api.raw_batch(batch)
    P = api.device_params(scene, batch)
    tuning = None
    if args.schedule is not None:
        dctx.set_launch(args.schedule, args.block, 0, args.adj_schedule if args.adj_schedule is not None
                        else args.schedule, args.adj_block or args.block, 0, args.adj_scatter)
    else:
        tuning = api.autotune(dctx, gs, adj, P, reps=1)
    lc = dctx.get_launch()

    # seeded target: the walls' and the diffuse sphere's albedo perturbed, other random numbers
    tp = scene.params()
    rng = np.random.default_rng(21)
    tp["tex"] = np.clip(tp["tex"] + rng.uniform(-0.15, 0.15, tp["tex"].shape), 0.05, 0.95)
    tp["theta"] = batch.theta
    tjobs = [copy.copy(j) for j in jobs]
    for j in tjobs:
        j.seed = 777
    target = api.render_primal(dctx, gs, api.pack_jobs(tjobs), api.device_params(scene, batch, tp)).clone()
    N = float(target.numel())
    stream = torch.cuda.Stream(device=dev)
    raw_buf = torch.empty(rb.image_floats, dtype=torch.float32, device=dev)
    loss_buf = torch.empty((), dtype=torch.float64, device=dev)
    grads = api.zero_grads(P)

    def step():
        # what PolarizedL2's forward and backward run, issued on one stream
        api.render_primal(dctx, gs, rb, P, image=raw_buf, stream=stream)
        api.loss_l2(dctx, gs, batch, P, raw_buf, rb.offsets, target, 1.0 / N, loss=loss_buf, stream=stream)
        for g in grads.values():
            g.zero_()
        api.render_adjoint_l2(dctx, gs, adj, P, raw_buf, rb.offsets, target, 1.0 / N, grads, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()                       # the library sizes its workspace here, before the capture
    stream.synchronize()
    dctx.sync_status(stream)
    dctx.stage_stats(timing=False, reset=True)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            graph.replay()
    stream.synchronize()

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with ClockSampler(clk_index) as clk:
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(K):
                flush.zero_()                    # L2 flush between timed replays (outside the events)
                ev[k][0].record(stream)
                graph.replay()
                ev[k][1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    dctx.sync_status(stream)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # per-kernel times: the same step run eagerly (the graph's kernels, launched one by one),
    # with the CUDA events the library records around each launch on the launching stream
    KS = min(K, 5)
    dctx.stage_stats(timing=True, reset=True)
    with torch.cuda.stream(stream):
        for _ in range(KS):
            flush.zero_()
            step()
    stream.synchronize()
    stages = dctx.stage_stats(timing=False, reset=True)
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    if args.kernels_only:
        # work units of one step's adjoint and primal passes and the number of steps the
        # process ran (warm-up, capture warm-up, timed, staged): what a profiler's per-launch
        # counters are divided by to give per-unit figures
        return {"value": weak_scaling_value(path_counts(jobs)[0], world, K, total_ms), "ms_per_step": total_ms / K,
                "stages": {k: v for k, v in stages.items() if v[0]}, "launch": list(lc),
                "steps_run": 2 * args.warmup + K + KS, "work_adjoint": api.count_work(dctx, gs, adj, P),
                "work_primal": api.count_work(dctx, gs, rb, P)}
    counted, traced = path_counts(jobs)
    value = weak_scaling_value(counted, world, K, total_ms)
    clocks = clk.summary()
    loss_val = float(loss_buf)

    # ---- the plain form: one render_primal + one render_adjoint per (view, angle)
    plain_jobs = []
    for j in jobs:
        for t in j.thetas:
            k = copy.copy(j)
            k.thetas = [t]
            plain_jobs.append(k)
    plain_batches = [api.pack_jobs([k]) for k in plain_jobs]
    plain_adj = [api.pack_jobs(api.adjoint_jobs([k])) for k in plain_jobs]
    views = api.image_views(batch, target)
    plain_targets = [views[vi][a].reshape(-1) for vi, j in enumerate(jobs) for a in range(j.num_angles)]
    plain_params = []
    for k in plain_jobs:
        q = dict(P)
        q["theta"] = torch.tensor([k.thetas[0]], dtype=torch.float32, device=dev)
        plain_params.append(q)
    pg = api.zero_grads(P)
    theta_scratch = torch.zeros(1, device=dev)

    def plain_all():
        for pb, pa, q, t in zip(plain_batches, plain_adj, plain_params, plain_targets):
            img = api.render_primal(dctx, gs, pb, q, stream=stream)
            d = (img - t).mul_(2.0 / N)
            gq = {"tex": pg["tex"], "ior": pg["ior"], "le": pg["le"], "sheet": pg["sheet"], "theta": theta_scratch}
            api.render_adjoint(dctx, gs, pa, q, d, gq, stream=stream)

    with torch.cuda.stream(stream):
        plain_all()                      # warm-up
    stream.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        flush.zero_()
        a.record(stream)
        plain_all()
        b.record(stream)
    b.synchronize()
    plain_ms = max_over_ranks(a.elapsed_time(b), world, dev)
    plain_traced = sum(2 * k.num_paths for k in plain_jobs)
    dctx.sync_status(stream)

    # ---- gradient memory of the autograd forms: peak device memory of forward + backward
    def peak(fn):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        fn()
        torch.cuda.synchronize()
        return torch.cuda.max_memory_allocated() - base

    leaf = {k: v.clone().requires_grad_(True) for k, v in P.items()}

    def batched_fused():
        api.PolarizedL2.apply(dctx, gs, batch, adj, target, leaf["tex"], leaf["ior"], leaf["le"], leaf["sheet"],
                              leaf["theta"]).backward()

    def batched_image():
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

    mem_fused = peak(batched_fused)
    mem_image = peak(batched_image)
    mem_plain = peak(plain_autograd)
    ws_batched = dctx.query_workspace(adj)
    ws_plain = max(dctx.query_workspace(pa) for pa in plain_adj[::NUM_ANGLES])

    # ---- end to end through the public autograd API, texture from and gradient to pinned host memory
    host_tex = torch.from_numpy(np.asarray(scene.params()["tex"], np.float32)).pin_memory()
    host_grad = torch.empty_like(host_tex).pin_memory()
    host_loss = torch.empty(1, dtype=torch.float32).pin_memory()
    tex_d = P["tex"].clone().requires_grad_(True)
    others = {k: P[k].clone().requires_grad_(True) for k in ("ior", "le", "sheet", "theta")}
    cur = torch.cuda.current_stream(dev)

    def e2e_step():
        tex_d.data.copy_(host_tex, non_blocking=True)
        tex_d.grad = None
        loss = api.PolarizedL2.apply(dctx, gs, batch, adj, target, tex_d, others["ior"], others["le"],
                                     others["sheet"], others["theta"])
        loss.backward()
        host_grad.copy_(tex_d.grad, non_blocking=True)
        host_loss.copy_(loss.detach().view(1), non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(K):
        flush.zero_()
        a.record(cur)
        e2e_step()
        b.record(cur)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e = {"value": weak_scaling_value(counted, world, K, e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": int(host_tex.numel() * 4), "d2h_bytes_per_step": int(host_grad.numel() * 4 + 4),
           "ms_per_step": e2e_ms / K, "api": "PolarizedL2.apply + loss.backward()"}

    # ---- roofline of the dominant kernel of the graph replays
    work = api.count_work(dctx, gs, adj, P)
    pwork = api.count_work(dctx, gs, rb, P)
    flops, cbytes = workload_flops(work, pwork, lc, KS)
    props = torch.cuda.get_device_properties(dev)
    roofline = roofline_of(stages, flops, cbytes, props, peaks, clocks, WORKLOAD, work)

    result = {
        "value": value, "ms_per_step": total_ms / K, "clocks": clocks,
        "config": {"workload": WORKLOAD if args.scale == 1.0 else f"{WORKLOAD} scaled {args.scale}",
                   "scene": "Cornell box: 12 triangles + 2 spheres, one quad light",
                   "views": [j.width for j in jobs], "angles": NUM_ANGLES, "spp": VIEW_SPP, "max_depth": VIEW_DEPTH,
                   "pixels": int(sum(j.num_pixels for j in jobs)),
                   "paths_counted_per_step": counted, "paths_traced_per_step": traced,
                   "paths_counted": "every (view, angle, pixel, sample) path of the primal and of the adjoint, "
                                    "as the plain form traces them; the batched form folds the angles exactly",
                   "step": "CUDA-graph replay of the batched fused-L2 gradient step (PolarizedL2 forward + backward "
                           "kernels: render_primal of all views, dppt_loss_l2, dppt_render_adjoint_l2)",
                   "grads": "albedo textures, IOR, emitter Stokes, 512 polarizer angles",
                   "l2": "flushed between timed steps (512 MiB write); the 2.9 GB target is read every step",
                   "schedule": {"primal": [api.SCHEDULE_NAMES[lc[0]], lc[1]],
                                "adjoint": [api.SCHEDULE_NAMES[lc[3]], lc[4]],
                                "adjoint_texel_scatter": ("warp", "lane")[lc[6]],
                                "chosen_by": "autotuner" if tuning else "command line"},
                   "parallelism": f"replicas{world}"},
        "batched": {"ms_per_step": total_ms / K, "paths_per_s": value,
                    "traced_paths_per_s": weak_scaling_value(traced, world, K, total_ms),
                    "p50_ms": statistics.median(step_ms), "p99_ms": sorted(step_ms)[min(K - 1, int(0.99 * K))],
                    "loss": loss_val,
                    "peak_autograd_bytes": int(mem_fused), "workspace_bytes": int(ws_batched),
                    "image_form_peak_autograd_bytes": int(mem_image)},
        "plain": {"calls": 2 * len(plain_jobs), "ms_per_step": plain_ms,
                  "paths_per_s": weak_scaling_value(counted, world, 1, plain_ms),
                  "traced_paths_per_s": weak_scaling_value(plain_traced, world, 1, plain_ms),
                  "peak_autograd_bytes": int(mem_plain), "workspace_bytes": int(ws_plain)},
        "vs_plain": {"paths_per_s": (total_ms / K) and plain_ms / (total_ms / K),
                     "gradient_mb_batched": mem_fused / 2**20, "gradient_mb_plain": mem_plain / 2**20,
                     "gradient_memory_ratio": mem_fused / max(1, mem_plain)},
        "stages": stage_report(stages, flops, cbytes, KS),
        "stages_note": f"per-kernel times over {KS} eager runs of the captured step (CUDA events the library "
                       "records around each launch on the launching stream); eager step "
                       f"{sum(v[1] for v in stages.values()) / KS:.2f} ms of kernel time",
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(sum(n for n, _ in stages.values()) / KS * K),
        "tuning": tuning,
    }
    return result


def run_icosphere(args, api, dctx, rank, dev, peaks):
    """The 50k-triangle icosphere gradient step (eager), its stages and dominant-kernel roofline."""
    import numpy as np
    import torch
    from paper_2607_13265_gb300 import scenegen as sg
    kw = {"width": max(8, int(round(256 * args.scale)))} if args.scale != 1.0 else {}
    scene, job = sg.icosphere_scene(**kw)
    job.stream = rank
    target_scene, tjob = sg.icosphere_scene(**kw)
    tp = target_scene.params()
    rng = np.random.default_rng(100)
    for t in (0, 1):
        off, w, h, ch = target_scene.tex_desc[t]
        lo, hi = ((0.2, 0.9), (0.05, 0.5))[t]
        tp["tex"][off:off + w * h * ch] = rng.uniform(lo, hi, w * h * ch)
    gs = api.GpuScene(dctx, scene)
    batch = api.pack_jobs([job])
    adj = api.pack_jobs(api.adjoint_jobs([job]))
    P = api.device_params(scene, batch)
    tuning = None
    if args.schedule is not None:
        dctx.set_launch(args.schedule, args.block, 0, args.adj_schedule if args.adj_schedule is not None
                        else args.schedule, args.adj_block or args.block, 0, args.adj_scatter)
    else:
        tuning = api.autotune(dctx, gs, adj, P, reps=2)
    lc = dctx.get_launch()
    tjob.seed = 12345
    target = api.render_primal(dctx, gs, api.pack_jobs([tjob]), api.device_params(scene, batch, tp)).clone()
    N = float(target.numel())
    grads = api.zero_grads(P)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        img = api.render_primal(dctx, gs, batch, P, stream=stream)
        dI = (img - target).mul_(2.0 / N)
        api.render_adjoint(dctx, gs, adj, P, dI, grads, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    dctx.stage_stats(timing=True, reset=True)
    for k in range(K):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    stages = dctx.stage_stats(timing=False, reset=True)
    dctx.sync_status()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    paths = 2 * job.num_paths
    work = api.count_work(dctx, gs, adj, P)
    pwork = api.count_work(dctx, gs, batch, P)
    flops, cbytes = workload_flops(work, pwork, lc, K)
    props = torch.cuda.get_device_properties(dev)
    fp = dctx.adjoint_footprint(job.max_depth)
    return {"workload": ICO_WORKLOAD, "paths_per_s": paths * K / (ms / 1000.0), "ms_per_step": ms / K,
            "paths_per_step": paths,
            "schedule": {"primal": [api.SCHEDULE_NAMES[lc[0]], lc[1]], "adjoint": [api.SCHEDULE_NAMES[lc[3]], lc[4]],
                         "adjoint_texel_scatter": ("warp", "lane")[lc[6]],
                         "chosen_by": "autotuner" if tuning else "command line"},
            "stages": stage_report(stages, flops, cbytes, K),
            "roofline": roofline_of(stages, flops, cbytes, props, peaks, {}, ICO_WORKLOAD, work),
            "memory": {"workspace_bytes": dctx.query_workspace(adj),
                       "prb_cache_bytes": (wave_paths([job]) * job.max_depth * WF_CACHE_FLOATS * 4 if lc[3] == 2
                                           else wave_paths([job]) * job.max_depth * SWEEP_RECORD_BYTES
                                           + fp["local_bytes_per_thread"] * fp["threads_per_sm"] * fp["sms"]
                                           if lc[3] == 3
                                           else fp["local_bytes_per_thread"] * fp["threads_per_sm"] * fp["sms"]),
                       "megakernel_local_bytes_per_thread": fp["local_bytes_per_thread"],
                       "megakernel_adjoint_registers": fp["registers"]},
            "gpu_launches": int(sum(n for n, _ in stages.values())),
            "tuning_times_ms": tuning["times_ms"] if tuning else None}


def run_native(args):
    import torch
    import torch.distributed as dist
    rank, world, local = _env_rank()
    pool = None
    cpu_procs = os.cpu_count() or 1
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.kernels_only:
        # the oracle's worker processes are spawned before the first CUDA call
        pool = mp.get_context("spawn").Pool(cpu_procs, initializer=_oracle_init, initargs=(args.scale,))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2607_13265_gb300 import api, build
    build.build()
    dev = torch.device("cuda", local)
    peaks = load_peaks()
    dctx = api.Context(local)
    if args.kernels_only:
        out = run_views(args, api, dctx, rank, world, dev, local, peaks) if args.only != "icosphere" else {}
        if not args.no_icosphere and args.only != "views":
            ico = run_icosphere(args, api, dctx, rank, dev, peaks)
            out["icosphere"] = {k: ico[k] for k in ("paths_per_s", "ms_per_step", "stages", "schedule")}
        if rank == 0:
            print(json.dumps(out))
        return
    views = run_views(args, api, dctx, rank, world, dev, local, peaks)
    ico = None if args.no_icosphere else run_icosphere(args, api, dctx, rank, dev, peaks)
    result = {
        "metric": METRIC, "value": views["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": views["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded procedural scene, textures and target)",
        "config": views["config"], "batched": views["batched"], "plain": views["plain"],
        "vs_plain": views["vs_plain"], "stages": views["stages"], "stages_note": views["stages_note"],
        "roofline": views["roofline"], "clocks": views["clocks"], "e2e": views["e2e"],
        "gpu_launches": views["gpu_launches"], "tuning": views["tuning"], "icosphere": ico,
    }
    if pool is not None:
        result["cpu_baseline"] = oracle_sample(args.cpu_pixels, cpu_procs, pool, args.scale)
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
    pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_init, initargs=(args.scale,))
    pool.map(_oracle_task, [(0, [0])] * procs)
    for _ in range(args.warmup):
        oracle_sample(args.ref_pixels, procs, pool, args.scale)
    walls, paths, traced = 0.0, 0, 0.0
    for _ in range(args.steps):
        r = oracle_sample(args.ref_pixels, procs, pool, args.scale)
        walls += r["wall_s"]
        paths += r["paths"]
    pool.close()
    pool.join()
    value = paths / walls
    sample = (f"{args.ref_pixels} evenly strided pixels over the 8 views of the {WORKLOAD} workload per step, "
              f"16 spp, all 64 angles (FP64 oracle: primal + cached-replay adjoint; paths counted as the "
              f"native arm counts them)")
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
    ap.add_argument("--steps", type=int, default=50, help="timed steps (graph replays: p50 and p99 over them)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--schedule", type=int, default=None,
                    help="0 grid, 1 persistent, 2 wavefront, 3 sweep (adjoint; its primal is the grid's) "
                         "(default: autotuner)")
    ap.add_argument("--block", type=int, default=128)
    ap.add_argument("--adj-schedule", type=int, default=None, help="adjoint schedule (default: same as --schedule)")
    ap.add_argument("--adj-block", type=int, default=None)
    ap.add_argument("--adj-scatter", type=int, default=0, choices=[0, 1],
                    help="with --schedule: texel gradients per warp group (0) or per lane (1)")
    ap.add_argument("--cpu-pixels", type=int, default=98304, help="pixels of the CPU-baseline sample")
    ap.add_argument("--ref-pixels", type=int, default=4096, help="pixels per step of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-icosphere", action="store_true")
    ap.add_argument("--scale", type=float, default=1.0, help="image sides scaled (tests and profiling captures only)")
    ap.add_argument("--kernels-only", action="store_true",
                    help="profiling captures: the timed steps only (no plain form, memory, end to end or CPU leg)")
    ap.add_argument("--only", choices=["views", "icosphere"], default=None,
                    help="with --kernels-only: one workload (--scale shrinks the icosphere's image too)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
