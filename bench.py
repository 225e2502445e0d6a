#!/usr/bin/env python3
"""Radio-map ray-bounces/s of the SBR tracer on B300.

One step = the radio maps of the largest workload: a procedural city of
0.97M triangles (210 x 210 extruded convex polygons, seed 5), 16
transmitters with 1e8 Fibonacci rays each, 28 GHz, up to 8 reflections /
refractions, 16 maps of 2048 x 2048 cells of 2 m, all in one persistent
launch.  The metric counts segments (closest-hit queries with their deposit
and shading) on the device.  The same line carries the adjoint over the
materials on that workload (its rate and forward+adjoint / forward; the
adjoint replays the closest hits the forward recorded, the re-tracing form
beside it), the end-to-end rate from host arrays, the roofline of the tracer
kernel and the FP64 oracle timed on the host; `extra` holds the Manhattan, batched and
differentiable workloads and the widened model, each with its roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank traces a city workload of its own: rank r takes
transmitters 16 r .. 16 r + 15 of one seeded draw of 16 N (the first 16 are
the one-GPU workload's).  Independent problems with fixed work per GPU, so no
collective is on the data path: weak scaling; the value is the segments of
all ranks over the slowest rank's time; rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import copy
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SEGMENT_BYTES = 184      # compulsory wavefront bytes per segment (ray state r/w, hit, queue)
SM_COUNT = 148           # set from the device in run_ours
METRIC = "radio-map ray-bounces/s"
UNIT = "ray-bounces/s"
WORKLOADS = {
    5: ("procedural city seed 5: 210x210 extruded convex 4-12-gon buildings (971006 triangles), 8 materials "
        "(ground half-space + 7 slab); 16 TX (seed 50, heights 10-50 m) x 1e8 Fibonacci rays, isotropic V-pol; "
        "28 GHz; max depth 8 (R+T); 16 maps of 2048x2048 cells of 2 m at z=1.5 m"),
    2: ("manhattan seed 2: 10x10 box buildings, 1202 triangles, 4 materials (ground half-space + 3 slab); "
        "1 TX at (0,0,30) m isotropic V-pol; 28 GHz; 1e7 Fibonacci rays; max depth 5 (R+T); "
        "512x512 map of 1 m cells at z=1.5 m"),
    3: ("manhattan seed 2, 64 TX (seed 3, heights 5-40 m) with 2^U(16,22) rays each; 28 GHz; max depth 3; "
        "64 maps of 256x256 cells of 2 m; one persistent CUDA-graph launch"),
    4: ("manhattan seed 4 (8 materials), 1 TX at (0,0,30) m, 1e6 rays, max depth 4, bilinear 256x256 map of "
        "2 m cells; dB-MSE loss against a map traced with seeded perturbed materials; adjoint over 8 eps_r, "
        "8 sigma and the TX position"),
}
# the committed ncu summaries a roofline's `traffic` comes from, keyed by workload
PROFILES = {5: "k_trace_city.md", 2: "k_trace_manhattan_1e7.md", 3: "k_trace_batched.md",
            4: "k_trace_adjoint_differentiable.md", "city_adjoint": "k_trace_adjoint_city.md",
            "city_adjoint_replay": "k_trace_adjoint_city_replay.md",
            "diffuse": "k_trace_diffuse_manhattan.md"}
# the tracer's code and the tree it walks (the BVH builders decide its node visits)
TRACE_SOURCES = [os.path.join(ROOT, "paper_2504_21719_b300", "csrc", f) for f in ("trace.cu", "common.cuh", "array.cuh", "bvh.cu")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--rays", type=int, default=0, help="override the rays per transmitter (profiling a smaller case)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- helpers
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def profiled(cfg, key: str):
    """A figure (dram_bytes_per_segment, issue_active_pct, ...) of a tracer
    workload from its committed ncu summary, if the kernel source is unchanged
    since it was taken; else None."""
    try:
        txt = open(os.path.join(ROOT, "profiles", PROFILES[cfg])).read()
    except (OSError, KeyError):
        return None
    h = hashlib.sha256()
    for p in TRACE_SOURCES:
        h.update(open(p, "rb").read())
    vals = {}
    for line in txt.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip().strip("-* `")] = v.strip().strip("` ")
    if vals.get("source_sha256") != h.hexdigest():
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def roofline(cfg, kernel: str, segments: float, kernel_ms: float, binding: str, timed_alone: bool):
    """HBM roofline of one tracer launch: 184 compulsory wavefront bytes per
    segment over the launch's CUDA-event duration, against the measured copy
    bandwidth; `traffic` = the committed ncu DRAM bytes per segment (of a
    capture of the same kernel) times this launch's segments."""
    pk = peaks()
    peak = pk.get("hbm_gbs")
    src = "measured" if peak else "fallback"
    peak = peak or 6400.0
    achieved = SEGMENT_BYTES * segments / (kernel_ms / 1e3) / 1e9
    per_seg = profiled(cfg, "dram_bytes_per_segment")
    issue = profiled(cfg, "issue_active_pct")
    # the limit that binds: warp instructions issued per second against the SMs' issue
    # peak (4 schedulers per SM, one instruction per cycle each, at the maximum SM clock);
    # instructions per segment from the committed full-size ncu count of this kernel
    wips = profiled(cfg, "warp_inst_per_segment")
    issue_roof = None
    if wips is not None and pk.get("sm_max_mhz"):
        ipeak = SM_COUNT * 4 * pk["sm_max_mhz"] * 1e6
        iach = wips * segments / (kernel_ms / 1e3)
        issue_roof = {"bound": "issue", "achieved": round(iach / 1e12, 4), "peak": round(ipeak / 1e12, 4),
                      "unit": "warp instructions/ns (1e12/s)", "frac": round(iach / ipeak, 4),
                      "warp_inst_per_segment": wips}
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None if per_seg is None else round(per_seg * segments),
            "peak_source": src, "algorithmic_bytes_per_segment": SEGMENT_BYTES, "kernel": kernel,
            "kernel_ms": round(kernel_ms, 4), "segments_per_launch": int(segments),
            "issue_slots_busy_frac": None if issue is None else round(issue / 100.0, 3),
            "binding_limit": binding, "peak_kind": "burst copy bandwidth" if timed_alone else "copy bandwidth",
            "issue_roofline": issue_roof}


def tuned(gpu_name: str, key: str):
    from paper_2504_21719_b300.autotune import lookup
    return lookup(gpu_name, key)


def tuned_params(api, p, gpu_name, key, **kw):
    blk, bps, qch, rfm = tuned(gpu_name, key)
    return api.params_from(p, block_size=blk, blocks_per_sm=bps, queue_chunk=qch, refill_min=rfm, **kw), \
        {"block_size": blk or 128, "blocks_per_sm": bps or "max occupancy", "queue_chunk": qch or 1,
         "refill_min": rfm or 20, "tuned": bool(blk)}


def oracle_sample(cfg: int, target_s: float = 12.0, record_segments=True):
    """The FP64 oracle, as it stands, on a bounded lattice subset of workload
    `cfg` (calibrated on a small subset, then sized to about target_s)."""
    import oracle
    from synth import scenes as S
    sc, txs, p = S.workload(cfg)

    def run(sub):
        t0 = time.perf_counter()
        segs = 0
        for tx in sub:
            r = oracle.radio_map(sc, tx, p, want_record=True)
            segs += int((r["record"][:, :, 0] != -2).sum())
        return segs, time.perf_counter() - t0

    def subset(stride, begin):
        out = []
        for t in txs:
            u = copy.copy(t)
            u.ray_stride, u.ray_begin = max(1, min(stride, t.num_rays)), begin % max(1, min(stride, t.num_rays))
            out.append(u)
        return out

    total = sum(t.num_rays for t in txs)
    # calibration: from about 1 in 10^4 of the rays (workload 5: one ray per
    # transmitter), growing the sample until it takes a measurable time
    cal = 100_000_000 if cfg == 5 else 10_000
    while True:
        segs, dt = run(subset(cal, 0))
        if dt >= 0.5 or cal <= 1 or cfg == 5:
            break
        cal = max(1, cal // 8)
    rays = sum(u.count() for u in subset(cal, 0))
    rate = rays / max(dt, 1e-3)
    want = max(rays, rate * target_s)
    stride = max(1, int(total / want))
    sub = subset(stride, 1)
    segs, dt = run(sub)
    n = sum(u.count() for u in sub)
    return {"value": round(segs / dt, 1), "unit": "segments/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"workload {cfg} lattice subset: 1 in {stride} rays of every transmitter ({n} rays, {segs} "
                      f"segments, {dt:.1f} s), FP64 brute force over {sc.nt} triangles, OpenMP"}


def traversal_counts(api, gs, txs, p, prm):
    """Node visits and triangle tests per segment, from one untimed trace with
    statistics on (the plain tracer does not count them)."""
    q = api.params_from(p, stats=True, block_size=prm.block_size, blocks_per_sm=prm.blocks_per_sm,
                        queue_chunk=prm.queue_chunk, refill_min=prm.refill_min)
    s = api.trace(gs, txs, q)["stats"]
    return s["nodes_visited"] / max(1, s["segments"]), s["tris_tested"] / max(1, s["segments"])


def time_plan(torch, plan, steps, warmup, flush, clocks=None):
    """Replay a graph-captured trace: warm-up, then `steps` timed launches with
    the L2 flushed before each; CUDA events around each launch on the current
    stream, the plan's own events around its tracer node."""
    for _ in range(warmup):
        plan.launch()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
        # nvidia-smi needs a moment to start sampling: keep the GPU busy meanwhile
        t_end = time.perf_counter() + 0.6
        while time.perf_counter() < t_end:
            plan.launch()
            torch.cuda.synchronize()
    step_ms, kern_ms, st = [], [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        flush.zero_()                         # L2 (126 MB) flushed between timed steps
        torch.cuda.synchronize()
        ev0.record()
        plan.launch()
        ev1.record()
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        s = plan.stats()
        kern_ms.append(s["kernel_ms"])
        st.append(s)
    clk = clocks.stop() if clocks is not None else None
    return step_ms, kern_ms, st, clk


def e2e_host(api, torch, sc, txs, prm, out, steps, warmup, flush, breakdown=0):
    """End to end through the public API from pinned host arrays: scene upload,
    BVH build (the default builder: binned SAH above 2048 triangles), trace and
    the read-back of the maps, every step.  With
    `breakdown` > 0, that many more steps time each part alone (synchronised
    after each)."""
    vh = torch.from_numpy(sc.verts).pin_memory()
    th = torch.from_numpy(sc.tris).pin_memory()
    mh = torch.from_numpy(sc.tri_mat).pin_memory()
    out_h = torch.empty(out.shape, dtype=torch.float32).pin_memory()
    e_ms, e_segs = [], []
    for i in range(warmup + steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = api.Scene(vh, th, mh, sc.mats)
        r = api.trace(g2, txs, prm, out=out)
        out_h.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        g2.free()
        if i >= warmup:
            e_ms.append(dt * 1e3)
            e_segs.append(r["stats"]["segments"])
    h2d = sc.verts.nbytes + sc.tris.nbytes + sc.tri_mat.nbytes + sc.mats.nbytes + 72 * len(txs) + 56
    res = {"value": sum(e_segs) / (sum(e_ms) / 1e3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(out_h.numel() * 4 + 576), "ms_per_step": round(statistics.mean(e_ms), 3),
           "includes": "scene upload + BVH build (binned SAH) + trace + map readback, per step"}
    if breakdown:
        parts = {"upload": [], "build": [], "trace_call": [], "trace_kernel": [], "readback": []}
        for i in range(warmup + breakdown):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g2 = api.Scene(vh, th, mh, sc.mats, build=False)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            g2.build_bvh()
            g2.info()                     # waits for the build to finish
            t2 = time.perf_counter()
            r = api.trace(g2, txs, prm, out=out)
            t3 = time.perf_counter()
            out_h.copy_(out, non_blocking=True)
            torch.cuda.synchronize()
            t4 = time.perf_counter()
            g2.free()
            if i >= warmup:
                parts["upload"].append(1e3 * (t1 - t0))
                parts["build"].append(1e3 * (t2 - t1))
                parts["trace_call"].append(1e3 * (t3 - t2))
                parts["trace_kernel"].append(r["stats"]["kernel_ms"])
                parts["readback"].append(1e3 * (t4 - t3))
        res["breakdown_ms"] = {k: round(statistics.median(v), 4) for k, v in parts.items()}
        res["breakdown_ms"]["note"] = ("each part synchronised alone; trace_call - trace_kernel = table copy, "
                                      "FP64 map clear, FP64->FP32 map, counters read-back and launch latency")
    return res


def over_ranks(dist, torch, ms, counts, device):
    """Whole-job figures of a multi-rank run: the slowest rank's time and the
    sums over ranks of the per-rank counts (segments, bytes)."""
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), [float(x) for x in c]


# ----------------------------------------------------------------------------- our arm
def run_ours(args, world, rank, local):
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2504_21719_b300 import api
    from synth import scenes as S

    gpu_name = torch.cuda.get_device_name(local)
    global SM_COUNT
    SM_COUNT = torch.cuda.get_device_properties(local).multi_processor_count
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # ---------------- the step: forward radio maps of the city workload ----------------
    sc, txs_all, p = S.workload(5)
    if world > 1:
        txs_all = S.city_transmitters(sc, 16 * world)
    if args.rays:
        for t in txs_all:
            t.num_rays = args.rays
    txs = txs_all[16 * rank:16 * (rank + 1)]     # this rank's workload
    prm, shape = tuned_params(api, p, gpu_name, "city")
    gs = api.Scene.from_obj(sc)
    maps = torch.empty((len(txs), p.ny, p.nx), dtype=torch.float32, device="cuda")
    plan = api.TracePlan(gs, txs, prm, maps)
    if dist:
        plan.launch()
        torch.cuda.synchronize()
        dist.barrier()
    step_ms, kern_ms, st, clk = time_plan(torch, plan, args.steps, args.warmup, flush, Clocks(local))
    plan.free()
    total_ms, total_segs = sum(step_ms), sum(s["segments"] for s in st)
    if dist:
        total_ms, (total_segs,) = over_ranks(dist, torch, total_ms, [total_segs], "cuda")
    value = total_segs / (total_ms / 1e3)
    seg_step = statistics.mean(s["segments"] for s in st)
    kavg = statistics.mean(kern_ms)
    nodes, tris = traversal_counts(api, gs, txs, p, prm)
    roof = roofline(5, "k_trace (persistent forward tracer), one launch over all transmitters", seg_step, kavg,
                    "instruction issue (rays stay in registers; the 109 MB scene is read from L2)", False)

    # ---------------- forward + adjoint over the materials, same workload ----------------
    adjoint = None
    if not args.no_adjoint:
        adjoint = city_adjoint(api, S, torch, sc, txs, p, prm, tuned_params(api, p, gpu_name, "city_adjoint")[0],
                               tuned_params(api, p, gpu_name, "city_adjoint_replay")[0], gs, kavg, seg_step)

    # ---------------- end to end from host arrays ----------------
    e2e = None
    if not args.no_e2e:
        e2e = e2e_host(api, torch, sc, txs, prm, maps, args.steps, 1, flush, breakdown=2)
        if dist:
            # every rank uploads the scene and reads back its own maps
            ms, (segs, h2d, d2h) = over_ranks(dist, torch, e2e["ms_per_step"],
                                              [e2e["value"] * e2e["ms_per_step"] / 1e3, e2e["h2d_bytes_per_step"],
                                               e2e["d2h_bytes_per_step"]], "cuda")
            e2e.update(value=segs / (ms / 1e3), ms_per_step=round(ms, 3), h2d_bytes_per_step=int(h2d),
                       d2h_bytes_per_step=int(d2h))
    gs.free()
    del maps

    extra = {}
    if not args.no_extra and rank == 0:
        extra = run_extra(api, S, torch, gpu_name, flush, args)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None
    cpu = None
    if world == 1 and not args.no_cpu_baseline and not args.rays:
        cpu = oracle_sample(5, 15.0)
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(statistics.mean(step_ms), 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[5], "transmitters": len(txs_all), "rays_per_tx": txs_all[0].num_rays,
                   "max_depth": p.max_depth, "map": [len(txs_all), p.ny, p.nx], "triangles": sc.nt,
                   "segments_per_step": int(seg_step), "nodes_per_segment": round(nodes, 2),
                   "tris_per_segment": round(tris, 2), **shape,
                   "l2": "flushed between timed steps (256 MB write)",
                   "step": "CUDA graph of one trace over all transmitters (map clear, k_trace, k_map_to_f32), replayed",
                   "parallelism": f"{world} rank(s), 16 transmitters each, no collective"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps,
        "clocks": clk, "adjoint": adjoint, "extra": extra,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return line


def city_adjoint(api, S, torch, sc, txs, p, prm, prm_adj, prm_rep, gs, fwd_kernel_ms, fwd_segments, reps=3):
    """Adjoint of the dB-MSE loss over the materials on the city workload: the
    target maps are traced with seeded perturbed materials, the loss gradient
    comes from the library's loss kernel, then the adjoint kernel is timed in
    its two forms: replaying the closest hits a recording forward kept (the
    line's value) and re-tracing the forward's rays through the BVH."""
    tgt_sc = S.Scene(sc.name, sc.verts, sc.tris, sc.tri_mat, S.perturb_materials(sc.mats, 40))
    gt = api.Scene.from_obj(tgt_sc)
    tgt = api.trace(gt, txs, prm)["maps"]
    gt.free()
    # the recording forward: the maps, plus the closest hit of every segment (4 B per ray
    # and depth on the device)
    fr = api.trace(gs, txs, prm, keep_hits=True)
    fk = fr["stats"]["kernel_ms"]
    hits = fr["hits"]
    loss, dL, valid = api.db_mse_loss(fr["maps"], tgt)
    del tgt, fr

    def timed(pa, **kw):
        api.grad(gs, txs, pa, dL, **kw)            # warm-up
        ks, segs = [], 0
        for _ in range(reps):
            a = api.grad(gs, txs, pa, dL, **kw)
            ks.append(a["stats"]["kernel_ms"])
            segs = a["stats"]["segments"]
        return statistics.mean(ks), segs

    r, segs = timed(prm_rep, hits=hits)
    hb = int(hits.numel()) * 4
    del hits
    k, _ = timed(prm_adj)
    return {"value": round(segs / (r / 1e3), 1), "unit": UNIT, "kernel_ms": round(r, 3), "segments": segs,
            "form": "replays the closest hit the recording forward kept for every segment (rm_radio_map_grad_hits)",
            "hits_bytes": hb, "recording_fwd_kernel_ms": round(fk, 3), "fwd_kernel_ms": round(fwd_kernel_ms, 3),
            "fwd_plus_adj_over_fwd": round((fk + r) / fwd_kernel_ms, 3),
            "loss_cells": int(valid), "parameters": "d loss / d(eps_r, sigma) of 8 materials",
            "roofline": roofline("city_adjoint_replay", "k_trace<adjoint> replaying recorded hits", segs, r,
                                 "instruction issue", False),
            "retrace": {"value": round(segs / (k / 1e3), 1), "unit": UNIT, "kernel_ms": round(k, 3),
                        "form": "re-traces the forward's rays through the BVH (rm_radio_map_grad)",
                        "fwd_plus_adj_over_fwd": round((fwd_kernel_ms + k) / fwd_kernel_ms, 3),
                        "roofline": roofline("city_adjoint", "k_trace<adjoint> (re-traces the forward's rays)", segs,
                                             k, "instruction issue", False)}}


def _kernel_rate(api, gs, txs, prm, reps=5):
    """Mean tracer kernel time (CUDA events inside the library) and segments/s."""
    for _ in range(2):
        api.trace(gs, txs, prm)
    ms, segs = [], 0
    for _ in range(reps):
        r = api.trace(gs, txs, prm)
        ms.append(r["stats"]["kernel_ms"])
        segs = r["stats"]["segments"]
    k = statistics.mean(ms)
    return {"value": round(segs / (k / 1e3), 1), "unit": UNIT, "kernel_ms": round(k, 3), "segments": segs}


def run_extra(api, S, torch, gpu_name, flush, args):
    """The Manhattan workload as a full line of its own, the batched 64-TX form,
    forward+adjoint of the differentiable workload, the widened model (diffuse
    reflection, early termination, synthetic arrays, diffraction, mesh
    surfaces) and the time-vs-N_S-and-N_A sweep on a street canyon."""
    import numpy as np

    out = {}
    deferred = []   # (entry, workload, seconds) of the CPU baselines, timed at the end
    # ---- Manhattan, 1e7 rays: graph step, roofline, end to end with its breakdown, oracle ----
    sc, txs, p = S.workload(2)
    prm, shape = tuned_params(api, p, gpu_name, "manhattan")
    gs = api.Scene.from_obj(sc)
    maps = torch.empty((1, p.ny, p.nx), dtype=torch.float32, device="cuda")
    plan = api.TracePlan(gs, txs, prm, maps)
    steps = max(args.steps, 10)
    step_ms, kern_ms, st, _ = time_plan(torch, plan, steps, max(args.warmup, 3), flush)
    plan.free()
    segs = statistics.mean(s["segments"] for s in st)
    km = statistics.mean(kern_ms)
    out["manhattan"] = {"workload": WORKLOADS[2], "value": round(sum(s["segments"] for s in st) / (sum(step_ms) / 1e3), 1),
                        "unit": UNIT, "ms_per_step": round(statistics.mean(step_ms), 4), "steps": steps,
                        "segments_per_step": int(segs), **shape,
                        "nodes_per_segment": round(traversal_counts(api, gs, txs, p, prm)[0], 2),
                        "roofline": roofline(2, "k_trace (persistent forward tracer)", segs, km,
                                             "instruction issue (scene and map stay in L1/L2)", True),
                        "e2e": e2e_host(api, torch, sc, txs, prm, maps, steps, 3, flush, breakdown=steps)}
    if not args.no_cpu_baseline:
        deferred.append((out["manhattan"], 2, 8.0))
    base = _kernel_rate(api, gs, txs, prm)
    # widened model on the same workload (same scene, TX, map)
    scd = sc.with_scattering(0.5, 0.2, np.arange(sc.nm) % 3, 3, 2, 0.6)
    pd = copy.copy(p)
    pd.diffuse = True
    gsd = api.Scene.from_obj(scd)
    d = _kernel_rate(api, gsd, txs, tuned_params(api, pd, gpu_name, "diffuse")[0])
    d["vs_specular"] = round(d["value"] / base["value"], 3)
    d["materials"] = "S = 0.5 on every material; ground Lambertian, buildings directive / backscattering"
    d["roofline"] = roofline("diffuse", "k_trace<diffuse>", d["segments"], d["kernel_ms"], "instruction issue", True)
    out["specular_same_call"] = base
    out["diffuse"] = d
    gsd.free()
    pr = copy.copy(p)
    pr.rr_depth, pr.rr_max_prob = 2, 0.5
    e = _kernel_rate(api, gs, txs, tuned_params(api, pr, gpu_name, "manhattan")[0])
    e["setting"] = "Russian roulette after 2 interactions, p_max = 0.5"
    out["early_termination"] = e
    ta = copy.copy(txs[0])
    ta.ant_pos, ta.precoding = S.uniform_linear_array(64, p.freq_hz, 0.5, axis=0)
    a = _kernel_rate(api, gs, [ta], prm)
    a["setting"] = "64-element half-wavelength ULA, uniform precoding"
    out["synthetic_array_64"] = a
    # first-order diffraction map of the same transmitter: 1200 wedges x 4096 samples
    wl = gs.wedges()
    pw = tuned_params(api, p, gpu_name, "diffraction")[0]
    for _ in range(2):
        api.diffraction_map(gs, txs, pw, 4096, wedges=wl)
    dk, dst = [], None
    for _ in range(5):
        r = api.diffraction_map(gs, txs, pw, 4096, wedges=wl)
        dk.append(r["stats"]["kernel_ms"])
        dst = r["stats"]
    k = statistics.mean(dk)
    out["diffraction"] = {"value": round(dst["rays"] / (k / 1e3), 1), "unit": "wedge samples/s",
                          "kernel_ms": round(k, 3), "samples": dst["rays"], "wedges": wl[1],
                          "in_map": dst["segments"], "deposits": dst["deposits"],
                          "setting": "4096 samples per wedge; two visibility queries and the UTD field per sample"}
    # the same map on a mesh measurement surface: 256 x 256 x 2 rolling-terrain triangles over the map
    sv, st_ = S.terrain_surface(256.0, 256)
    su = api.surface(sv, st_)
    for _ in range(2):
        api.trace_mesh(gs, su, txs, prm)
    mk, mst = [], None
    for _ in range(5):
        r = api.trace_mesh(gs, su, txs, prm)
        mk.append(r["stats"]["kernel_ms"])
        mst = r["stats"]
    k = statistics.mean(mk)
    out["mesh_surface"] = {"value": round(mst["segments"] / (k / 1e3), 1), "unit": UNIT, "kernel_ms": round(k, 3),
                           "segments": mst["segments"], "crossings": mst["deposits"], "cells": int(len(st_)),
                           "setting": "one cell per triangle of a 131072-triangle terrain mesh over the map"}
    for _ in range(2):
        api.diffraction_map_mesh(gs, su, txs, p, 4096, wedges=wl)
    dk, dst = [], None
    for _ in range(5):
        r = api.diffraction_map_mesh(gs, su, txs, p, 4096, wedges=wl)
        dk.append(r["stats"]["kernel_ms"])
        dst = r["stats"]
    k = statistics.mean(dk)
    out["diffraction_mesh_surface"] = {"value": round(dst["rays"] / (k / 1e3), 1), "unit": "wedge samples/s",
                                       "kernel_ms": round(k, 3), "samples": dst["rays"], "deposits": dst["deposits"],
                                       "setting": "4096 samples per wedge onto the same terrain mesh"}
    su.free()
    gs.free()

    # ---- batched: 64 TX with uneven ray counts in one graph-captured persistent launch ----
    # (one static scene traced by every transmitter: the binned-SAH tree, which the default
    # builder keeps for meshes above 2048 triangles, saves 5 % of the launch for a 0.4 ms build)
    sc, txs, p = S.workload(3)
    gs = api.Scene.from_obj(sc, builder="sah")
    prm, shape = tuned_params(api, p, gpu_name, "batched")
    maps = torch.empty((len(txs), p.ny, p.nx), dtype=torch.float32, device="cuda")
    plan = api.TracePlan(gs, txs, prm, maps)
    step_ms, kern_ms, st, _ = time_plan(torch, plan, 5, 3, flush)
    plan.free()
    segs = st[-1]["segments"]
    out["batched_64tx"] = {"workload": WORKLOADS[3], "value": round(segs / (statistics.mean(step_ms) / 1e3), 1),
                           "unit": UNIT, "ms_per_launch": round(statistics.mean(step_ms), 3), "segments": segs,
                           "rays": sum(t.num_rays for t in txs), "form": "CUDA graph, one persistent launch",
                           "builder": "sah", **shape,
                           "roofline": roofline(3, "k_trace (one launch over 64 transmitters)", segs,
                                                statistics.mean(kern_ms), "instruction issue", True)}
    if not args.no_cpu_baseline:
        deferred.append((out["batched_64tx"], 3, 8.0))
    gs.free()

    # ---- differentiable: forward, dB loss, adjoint ----
    sc, txs, p = S.workload(4)
    gs = api.Scene.from_obj(sc)
    tgt_sc = S.Scene(sc.name, sc.verts, sc.tris, sc.tri_mat, S.perturb_materials(sc.mats, 40))
    gt = api.Scene.from_obj(tgt_sc)
    tgt = api.trace(gt, txs, p)["maps"][0]
    gt.free()
    pf = tuned_params(api, p, gpu_name, "manhattan")[0]
    pa = tuned_params(api, p, gpu_name, "adjoint")[0]
    par = tuned_params(api, p, gpu_name, "adjoint_replay")[0]
    f_ms, a_ms, b_ms, segs = [], [], [], 0
    for i in range(13):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = api.trace(gs, txs, pf)
        loss, dL, _ = api.db_mse_loss(f["maps"][0], tgt)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        a = api.grad(gs, txs, pa, dL.view(1, p.ny, p.nx))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if i >= 3:
            f_ms.append(f["stats"]["kernel_ms"])
            a_ms.append(a["stats"]["kernel_ms"])
            segs = f["stats"]["segments"]
            b_ms.append((t2 - t1) * 1e3)
    fk, ak = statistics.mean(f_ms), statistics.mean(a_ms)
    # the same step with the forward recording its hits and the adjoint replaying them
    rf_ms, ra_ms = [], []
    for i in range(8):
        f = api.trace(gs, txs, pf, keep_hits=True)
        loss, dL, _ = api.db_mse_loss(f["maps"][0], tgt)
        a = api.grad(gs, txs, par, dL.view(1, p.ny, p.nx), hits=f["hits"])
        if i >= 3:
            rf_ms.append(f["stats"]["kernel_ms"])
            ra_ms.append(a["stats"]["kernel_ms"])
    rfk, rak = statistics.mean(rf_ms), statistics.mean(ra_ms)
    out["differentiable"] = {"workload": WORKLOADS[4], "fwd_kernel_ms": round(fk, 3), "adj_kernel_ms": round(ak, 3),
                             "fwd_plus_adj_over_fwd": round((fk + ak) / fk, 3),
                             "adj_call_ms": round(statistics.median(b_ms), 3),
                             "fwd_plus_adj_call_over_fwd": round((fk + statistics.median(b_ms)) / fk, 3),
                             "fwd_value": round(segs / (fk / 1e3), 1), "adj_value": round(segs / (ak / 1e3), 1),
                             "unit": UNIT, "segments": segs,
                             "roofline_fwd": roofline(0, "k_trace<bilinear>", segs, fk, "instruction issue", True),
                             "roofline_adj": roofline(4, "k_trace<adjoint, bilinear>", segs, ak, "instruction issue", True),
                             "replay": {"recording_fwd_kernel_ms": round(rfk, 3), "adj_kernel_ms": round(rak, 3),
                                        "adj_value": round(segs / (rak / 1e3), 1), "unit": UNIT,
                                        "fwd_plus_adj_over_fwd": round((rfk + rak) / fk, 3),
                                        "form": "the adjoint replays the closest hits the forward recorded"}}
    if not args.no_cpu_baseline:
        deferred.append((out["differentiable"], 4, 6.0))
    gs.free()
    # the same with diffuse reflection on every material (adjoint kernel timed inside the library)
    scd = sc.with_scattering(np.linspace(0.2, 0.8, sc.nm), 0.3, np.arange(sc.nm) % 3, 2, 3, 0.5)
    pd = copy.copy(p)
    pd.diffuse = True
    gs = api.Scene.from_obj(scd)
    fk, ak = [], []
    for i in range(6):
        f = api.trace(gs, txs, pd)
        a = api.grad(gs, txs, pd, torch.ones_like(f["maps"]))
        if i >= 2:
            fk.append(f["stats"]["kernel_ms"])
            ak.append(a["stats"]["kernel_ms"])
    rk, rak = [], []
    for i in range(6):
        f = api.trace(gs, txs, pd, keep_hits=True)
        a = api.grad(gs, txs, pd, torch.ones_like(f["maps"]), hits=f["hits"])
        if i >= 2:
            rk.append(f["stats"]["kernel_ms"])
            rak.append(a["stats"]["kernel_ms"])
    out["differentiable_diffuse"] = {"fwd_kernel_ms": round(statistics.mean(fk), 3),
                                     "adj_kernel_ms": round(statistics.mean(ak), 3),
                                     "fwd_plus_adj_over_fwd": round(1 + statistics.mean(ak) / statistics.mean(fk), 3),
                                     "replay": {"recording_fwd_kernel_ms": round(statistics.mean(rk), 3),
                                                "adj_kernel_ms": round(statistics.mean(rak), 3),
                                                "fwd_plus_adj_over_fwd": round((statistics.mean(rk) + statistics.mean(rak))
                                                                               / statistics.mean(fk), 3)}}
    gs.free()
    out["time_vs_samples_and_antennas"] = sweep_samples_antennas(api, S, torch, gpu_name)
    # the oracle's OpenMP worker threads slow this process's later host calls by ~0.3-0.5 ms
    # each, so the CPU baselines run after every GPU measurement
    for entry, cfg, secs in deferred:
        entry["cpu_baseline"] = oracle_sample(cfg, secs)
    return out


def sweep_samples_antennas(api, S, torch, gpu_name, n_s=(10**6, 10**7, 10**8, 10**9), n_a=(1, 16, 128, 1024)):
    """Radio-map time of one transmitter 20 m above a street canyon as the number of
    samples N_S and of transmit-array elements N_A grow (the timing study of
    Sec. 4.4): depth 5, 3.5 GHz, 256 x 256 cells of 1 m, half-wavelength ULA with
    uniform precoding (N_A = 1: a single antenna).  Kernel time and the wall time
    of the `trace()` call, milliseconds, medians of two calls after one warm-up."""
    sc = S.street_canyon()
    gs = api.Scene.from_obj(sc)
    p = S.TraceParams(3.5e9, 5, cell_size=1.0, nx=256, ny=256)
    prm, _ = tuned_params(api, p, gpu_name, "manhattan")
    kern, call, segs = [], [], []
    for ns in n_s:
        kr, cr, sr = [], [], []
        for na in n_a:
            tx = S.Tx(pos=(0.0, 0.0, 20.0), num_rays=ns, seed=11)
            if na > 1:
                tx.ant_pos, tx.precoding = S.uniform_linear_array(na, p.freq_hz, 0.5)
            km, cm = [], []
            for i in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = api.trace(gs, [tx], prm)
                torch.cuda.synchronize()
                if i:
                    cm.append((time.perf_counter() - t0) * 1e3)
                    km.append(r["stats"]["kernel_ms"])
            kr.append(round(statistics.median(km), 3))
            cr.append(round(statistics.median(cm), 3))
            sr.append(r["stats"]["segments"])
            del r
        kern.append(kr)
        call.append(cr)
        segs.append(sr)
    gs.free()
    return {"scene": sc.name, "triangles": sc.nt, "N_S": list(n_s), "N_A": list(n_a),
            "kernel_ms": kern, "call_ms": call, "segments": segs,
            "setting": "TX 20 m above the street, depth 5, 3.5 GHz, 256 x 256 x 1 m map, ULA along y"}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    """The FP64 oracle on the host cores: each step a bounded lattice sample of
    the city workload (one transmitter per step, in turn)."""
    if rank != 0:
        return None
    import oracle
    from synth import scenes as S
    sc, txs, p = S.workload(5)
    stride = 4_000_000                             # 25 rays of one transmitter per step
    times, segs = [], []
    for i in range(args.warmup + args.steps):
        tx = copy.copy(txs[i % len(txs)])
        tx.ray_stride, tx.ray_begin = stride, (7 * i) % stride
        t0 = time.perf_counter()
        r = oracle.radio_map(sc, tx, p, want_record=True)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            segs.append(int((r["record"][:, :, 0] != -2).sum()))
    value = sum(segs) / sum(times)
    sample = (f"per step: 1 in {stride} rays of one transmitter's 1e8-ray lattice (25 rays, the transmitters in "
              f"turn), FP64 brute force over {sc.nt} triangles, OpenMP")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(times), 2),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[5], "sampled": True},
            "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return line


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
