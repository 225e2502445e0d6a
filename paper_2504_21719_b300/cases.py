"""Run one workload of the library a few times, for profilers and timing.

    python -m paper_2504_21719_b300.cases CASE [--rays N] [--reps R] [--builder auto|lbvh|sah]

CASE is one of
  manhattan    forward trace, Manhattan scene (1202 triangles), 1 TX, depth 5
  diffuse      the same with diffuse reflection on every material (S = 0.5)
  adjoint      adjoint of the differentiable workload (8 materials, bilinear)
  diffraction  first-order diffraction map, Manhattan, 1200 wedges
  city         forward trace, 0.97M-triangle procedural city, 1 TX, 1e7 rays, depth 8
  city_adjoint forward then adjoint (uniform dL/dC) of the same city trace; with
               --replay the forward records its hits and the adjoint replays them
  batched      the 64-TX batched workload (depth 3) in one launch on the binned-SAH tree
               (as the benchmark); --rays sets the lattice stride of every transmitter
               (default 1: the full workload)
  mesh         the Manhattan trace on a 131072-triangle terrain measurement surface
  diffraction_mesh  the diffraction map onto the same terrain surface (1200 wedges)
  array        the timing study's street canyon (depth 5, 3.5 GHz) from one transmitter with
               a 1024-element uniform linear array, 1e7 rays (the array factor's pre-pass
               kernel, then the tracer)
Each case runs in the launch shape the tuning table holds for its workload
class on this GPU (the benchmark's shape) and prints one line: case, kernel
ms of the last call, and its work counters.
"""
from __future__ import annotations

import argparse
import copy


def main(argv=None):
    import numpy as np
    import torch

    from . import api
    from synth import scenes as S

    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["manhattan", "diffuse", "adjoint", "diffraction", "city", "city_adjoint",
                                    "batched", "mesh", "array", "diffraction_mesh"])
    ap.add_argument("--rays", type=int, default=0, help="rays per TX (trace cases) or samples per wedge")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--builder", default="auto", choices=["auto", "lbvh", "sah"], help="the scene's BVH builder")
    ap.add_argument("--replay", action="store_true", help="adjoint cases: replay the forward's recorded hits")
    a = ap.parse_args(argv)
    if a.case in ("manhattan", "diffuse", "diffraction", "mesh", "diffraction_mesh"):
        sc, txs, p = S.workload(2)
        if a.case == "diffuse":
            sc = sc.with_scattering(0.5, 0.2, np.arange(sc.nm) % 3, 3, 2, 0.6)
            p = copy.copy(p)
            p.diffuse = True
    elif a.case in ("city", "city_adjoint"):
        sc, txs, p = S.workload(5)
        txs = txs[:1]
        txs[0].num_rays = 10_000_000
    elif a.case == "array":
        sc = S.street_canyon()
        p = S.TraceParams(3.5e9, 5, cell_size=1.0, nx=256, ny=256)
        txs = [S.Tx(pos=(0.0, 0.0, 20.0), num_rays=10_000_000, seed=11)]
        txs[0].ant_pos, txs[0].precoding = S.uniform_linear_array(1024, p.freq_hz, 0.5)
    elif a.case == "batched":
        sc, txs, p = S.workload(3)
        for t in txs:
            t.ray_stride = max(1, a.rays)
    else:
        sc, txs, p = S.workload(4)
    if a.rays and a.case not in ("diffraction", "diffraction_mesh", "batched"):
        txs[0].num_rays = a.rays
    from .autotune import lookup
    cls = {"manhattan": "manhattan", "diffuse": "diffuse", "adjoint": "adjoint", "diffraction": "diffraction",
           "city": "city", "city_adjoint": "city_adjoint", "batched": "batched", "mesh": "manhattan",
           "array": "manhattan", "diffraction_mesh": "diffraction"}[a.case]
    if a.replay and a.case in ("adjoint", "city_adjoint"):
        cls += "_replay"
    blk, bps, qch, rfm = lookup(torch.cuda.get_device_name(0), cls)
    p = api.params_from(p, block_size=blk, blocks_per_sm=bps, queue_chunk=qch, refill_min=rfm)
    builder = "sah" if (a.case == "batched" and a.builder == "auto") else a.builder
    gs = api.Scene.from_obj(sc, builder=builder)
    su = api.surface(*S.terrain_surface(256.0, 256)) if a.case in ("mesh", "diffraction_mesh") else None
    for _ in range(a.reps):
        if a.case == "mesh":
            r = api.trace_mesh(gs, su, txs, p)
        elif a.case == "diffraction_mesh":
            r = api.diffraction_map_mesh(gs, su, txs, p, a.rays or 4096)
        elif a.case == "diffraction":
            r = api.diffraction_map(gs, txs, p, a.rays or 4096)
        elif a.case in ("adjoint", "city_adjoint"):
            f = api.trace(gs, txs, p, keep_hits=a.replay)
            r = api.grad(gs, txs, p, torch.ones_like(f["maps"]), hits=f.get("hits"))
        else:
            r = api.trace(gs, txs, p)
    torch.cuda.synchronize()
    st = r["stats"]
    print(a.case, "kernel_ms", round(st["kernel_ms"], 4), "rays", st["rays"], "segments", st["segments"],
          "deposits", st["deposits"])
    if su is not None:
        su.free()
    gs.free()


if __name__ == "__main__":
    main()
