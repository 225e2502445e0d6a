"""Autotuner of the tracer's launch shape.

For each workload class it times, with the tracer's own CUDA-event timing
(rm_stats.kernel_ms), a staged search:
  1. the launch shape: block size (threads per block), resident blocks per SM
     (persistent grid size) and work-queue chunk (items a warp takes per queue
     access, in units of 32), at refill threshold 24;
  2. on the best shape, every refill threshold (idle lanes a warp waits for
     before it takes new rays);
and keeps the fastest.  The classes are the forward tracer on the Manhattan
workload, the batched 64-TX launch, the city, the diffuse forward, the adjoint
(differentiable workload and city, re-tracing and replaying recorded hits)
and the diffraction kernel (block size only).  Results go to tuning.json keyed by GPU name and class; bench.py and
callers read them back with ``lookup``.

    python -m paper_2504_21719_b300.autotune            # tunes and writes tuning.json
"""
from __future__ import annotations

import json
import os
import statistics

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning.json")

BLOCKS = (128, 256)
BLOCKS_PER_SM = (0, 2, 3, 4, 6)   # 0 = as many as fit
CHUNKS = (1, 4)
REFILLS = (8, 12, 16, 20, 22, 24, 26, 28, 30, 32)
# the library's defaults (rm_trace_params fields left at 0)
DEFAULT = {"block_size": 128, "blocks_per_sm": 0, "queue_chunk": 1, "refill_min": 20}


def lookup(gpu_name: str, key: str):
    """(block_size, blocks_per_sm, queue_chunk, refill_min) for a workload class,
    or zeros (library defaults)."""
    try:
        t = json.load(open(TABLE))
    except (OSError, ValueError):
        return 0, 0, 0, 0
    e = t.get(gpu_name, {}).get(key) or t.get("default", {}).get(key)
    if not e:
        return 0, 0, 0, 0
    return (int(e["block_size"]), int(e["blocks_per_sm"]), int(e.get("queue_chunk", 0)),
            int(e.get("refill_min", 0)))


def _time(run, reps):
    run()                                          # warm-up
    return statistics.median(run() for _ in range(reps))


def tune(api, scene, txs, params_obj, reps: int = 5, adjoint: bool = False, replay: bool = False):
    """Staged search over the launch shape, then the refill threshold; returns
    (best, all results, the library defaults' time).  replay: the adjoint
    replaying the hits of one recording forward."""
    import torch
    g = hits = None
    if adjoint:
        f = api.trace(scene, txs, params_obj, keep_hits=replay)
        g = torch.full_like(f["maps"], 1e-6)
        hits = f.get("hits")
        del f

    def run_with(cfg):
        p = api.params_from(params_obj, **cfg)
        if adjoint:
            return lambda: api.grad(scene, txs, p, g, hits=hits)["stats"]["kernel_ms"]
        return lambda: api.trace(scene, txs, p)["stats"]["kernel_ms"]

    results = []
    for blk in BLOCKS:
        for bps in BLOCKS_PER_SM:
            if bps and blk * bps > 2048:
                continue
            for ch in CHUNKS:
                cfg = {"block_size": blk, "blocks_per_sm": bps, "queue_chunk": ch, "refill_min": 24}
                results.append({**cfg, "kernel_ms": _time(run_with(cfg), reps)})
    shape = min(results, key=lambda e: e["kernel_ms"])
    for rf in REFILLS:
        cfg = {k: shape[k] for k in ("block_size", "blocks_per_sm", "queue_chunk")}
        cfg["refill_min"] = rf
        results.append({**cfg, "kernel_ms": _time(run_with(cfg), reps)})
    best = min(results, key=lambda e: e["kernel_ms"])
    default_ms = _time(run_with(DEFAULT), reps)
    return best, results, default_ms


def tune_diffraction(api, scene, txs, params_obj, samples=4096, reps=5):
    """Block size of the diffraction kernel (its grid is sized from it)."""
    wl = scene.wedges()
    res = []
    for blk in (64, 128, 192, 256):
        p = api.params_from(params_obj, block_size=blk)
        run = lambda: api.diffraction_map(scene, txs, p, samples, wedges=wl)["stats"]["kernel_ms"]
        res.append({"block_size": blk, "blocks_per_sm": 0, "kernel_ms": _time(run, reps)})
    best = min(res, key=lambda e: e["kernel_ms"])
    default = next(r for r in res if r["block_size"] == 256)
    return best, res, default["kernel_ms"]


def main(argv=None):
    import argparse
    import copy

    import numpy as np
    import torch

    from . import api
    import synth.scenes as S

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--only", default="", help="comma-separated classes (default: all)")
    a = ap.parse_args(argv)
    name = torch.cuda.get_device_name(0)
    try:
        table = json.load(open(TABLE))
    except (OSError, ValueError):
        table = {}
    entry = table.setdefault(name, {})
    sc2, txs2, p2 = S.workload(2)
    scd = sc2.with_scattering(0.5, 0.2, np.arange(sc2.nm) % 3, 3, 2, 0.6)
    pd = copy.copy(p2)
    pd.diffuse = True
    sc5, txs5, p5 = S.workload(5)
    # the city is tuned on one transmitter with 1e7 rays (the shape, not the size, is tuned)
    t5 = copy.copy(txs5[0])
    t5.num_rays = 10_000_000
    jobs = {"manhattan": (sc2, txs2, p2, False), "batched": (*S.workload(3), False),
            "city": (sc5, [t5], p5, False), "city_adjoint": (sc5, [t5], p5, True),
            "city_adjoint_replay": (sc5, [t5], p5, True), "diffuse": (scd, txs2, pd, False),
            "adjoint": (*S.workload(4), True), "adjoint_replay": (*S.workload(4), True)}
    only = [k for k in a.only.split(",") if k]
    for key, (sc, txs, p, adj) in jobs.items():
        if only and key not in only:
            continue
        gs = api.Scene.from_obj(sc, builder="sah" if key == "batched" else "auto")   # the benchmark's trees
        best, res, dflt = tune(api, gs, txs, p, adjoint=adj, replay=key.endswith("_replay"))
        entry[key] = {**best, "default_kernel_ms": dflt, "gain_over_default": round(dflt / best["kernel_ms"], 4),
                      "candidates": len(res)}
        gs.free()
        print(key, entry[key], flush=True)
    if not only or "diffraction" in only:
        gs = api.Scene.from_obj(sc2)
        best, res, dflt = tune_diffraction(api, gs, txs2, p2)
        entry["diffraction"] = {**best, "default_kernel_ms": dflt,
                                "gain_over_default": round(dflt / best["kernel_ms"], 4), "candidates": len(res)}
        gs.free()
        print("diffraction", entry["diffraction"], flush=True)
    json.dump(table, open(a.out, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
