"""Autotuner of the tracer's launch shape.

For a workload it times every combination of block size (threads per block),
resident blocks per SM (persistent grid size), work-queue chunk (items a
warp takes per queue access, in units of 32) and refill threshold (idle lanes
a warp waits for before it takes new rays) with the tracer's own CUDA-event
timing (rm_stats.kernel_ms) and keeps the fastest.  Results go to
tuning.json keyed by GPU name and workload class; bench.py and callers read
them back with ``lookup``.

    python -m paper_2504_21719_b300.autotune            # tunes and writes tuning.json
"""
from __future__ import annotations

import json
import os
import statistics

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning.json")

BLOCKS = (128, 256)
BLOCKS_PER_SM = (0, 2, 3, 4, 6, 8)   # 0 = as many as fit
CHUNKS = (1, 4)
REFILLS = (1, 8, 16, 20, 24, 28)


def lookup(gpu_name: str, key: str):
    """(block_size, blocks_per_sm, queue_chunk, refill_min) for a workload class, or
    zeros (library defaults)."""
    try:
        t = json.load(open(TABLE))
    except (OSError, ValueError):
        return 0, 0, 0, 0
    e = t.get(gpu_name, {}).get(key) or t.get("default", {}).get(key)
    if not e:
        return 0, 0, 0, 0
    return (int(e["block_size"]), int(e["blocks_per_sm"]), int(e.get("queue_chunk", 0)),
            int(e.get("refill_min", 0)))


def tune(api, scene, txs, params_obj, reps: int = 5, blocks=BLOCKS, bps_list=BLOCKS_PER_SM, chunks=CHUNKS,
         refills=REFILLS):
    """Time every launch shape; returns (best, all results)."""
    results = []
    for blk in blocks:
        for bps in bps_list:
            if bps and blk * bps > 2048:
                continue
            for ch in chunks:
                for rf in refills:
                    p = api.params_from(params_obj, block_size=blk, blocks_per_sm=bps, queue_chunk=ch,
                                        refill_min=rf)
                    r = api.trace(scene, txs, p)          # warm-up
                    ms = [api.trace(scene, txs, p)["stats"]["kernel_ms"] for _ in range(reps)]
                    results.append({"block_size": blk, "blocks_per_sm": bps, "queue_chunk": ch, "refill_min": rf,
                                    "kernel_ms": statistics.median(ms), "segments": r["stats"]["segments"]})
    best = min(results, key=lambda e: e["kernel_ms"])
    return best, results


def main(argv=None):
    import argparse

    import torch

    from . import api
    import synth.scenes as S

    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    out = ap.parse_args(argv).out
    name = torch.cuda.get_device_name(0)
    try:
        table = json.load(open(TABLE))
    except (OSError, ValueError):
        table = {}
    entry = table.setdefault(name, {})
    jobs = {"manhattan": S.workload(2), "batched": S.workload(3)}
    sc5, txs5, p5 = S.workload(5)
    # the city is tuned on one transmitter with 1e7 rays (the shape, not the size, is tuned)
    t5 = txs5[0]
    t5.num_rays = 10_000_000
    jobs["city"] = (sc5, [t5], p5)
    for key, (sc, txs, p) in jobs.items():
        gs = api.Scene.from_obj(sc)
        best, res = tune(api, gs, txs, p)
        base = next(r for r in res if r["block_size"] == 128 and r["blocks_per_sm"] == 0 and r["queue_chunk"] == 1
                    and r["refill_min"] == 20)
        entry[key] = {**best, "default_kernel_ms": base["kernel_ms"], "candidates": len(res)}
        gs.free()
        print(key, entry[key], flush=True)
    json.dump(table, open(out, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
