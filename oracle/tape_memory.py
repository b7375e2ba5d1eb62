"""Memory model of conventional reverse AD ("Conv. AD", Sec. 5.1) on the deep-path
workload -- TEST INFRASTRUCTURE, run by hand; it calls only this package.

Conventional AD keeps, for every path, the tape of every parameter-dependent scalar
operation of the whole path until the reverse sweep.  The oracle's taped route records
exactly those operations (one Wengert-list node each: two operand indices and two local
partials), so its node count is the tape a conventional implementation needs.  Here it is
counted on a uniform sample of the deep_stack_scene image (the full workload's view and
path mix at fewer pixels), then scaled to 1280 x 720 x 1 spp at
  * 16 B per node (FP32 partials + 32-bit operand indices, the tape's own layout), and
  * 4 B per node (a single FP32 value: a lower bound for any tape).
Cached suffix replay keeps 31 floats (124 B) per vertex of the path instead.

    python -m oracle.tape_memory [--depths 4 8 16 32 64 128] [--width 64 --height 36]
prints one JSON line per depth.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import OracleScene, stats


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--depths", type=int, nargs="+", default=[4, 8, 16, 32, 64, 128])
    ap.add_argument("--width", type=int, default=64)
    ap.add_argument("--height", type=int, default=36)
    args = ap.parse_args(argv)
    from paper_2607_13265_gb300 import scenegen as sg
    full_paths = 1280 * 720
    out = []
    for d in args.depths:
        scene, job = sg.deep_stack_scene(width=args.width, height=args.height, spp=1, depth=d)
        o = OracleScene(scene)
        img = o.render(job, scene.params())
        dI = np.random.default_rng(0).normal(size=img.shape)
        stats(reset=True)
        t0 = time.time()
        o.gradient(job, scene.params(), dI, mode="tape")
        st = stats(reset=True)
        paths = job.width * job.height * job.spp
        nodes_per_path = st["tape_total_nodes"] / paths
        vertices_per_path = st["vertices"] / paths
        row = {"depth": d, "sample_paths": paths, "vertices_per_path": vertices_per_path,
               "tape_nodes_per_path": nodes_per_path,
               "tape_nodes_per_vertex": nodes_per_path / max(vertices_per_path, 1e-30),
               "conv_ad_bytes_16B": nodes_per_path * full_paths * 16,
               "conv_ad_bytes_4B_lower_bound": nodes_per_path * full_paths * 4,
               "cache_bytes_full": vertices_per_path * full_paths * 124,
               "oracle_s": time.time() - t0}
        out.append(row)
        print(json.dumps(row))
    return out


if __name__ == "__main__":
    main()
