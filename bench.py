#!/usr/bin/env python3
"""Radio-map ray-bounces/s of the SBR tracer on B300.

One step = one full radio map of the Manhattan workload: 10 x 10 box
buildings (1202 triangles, seed 2), one transmitter at (0, 0, 30) m, 28 GHz,
1e7 Fibonacci rays, up to 5 reflections / refractions, 512 x 512 cells of
1 m.  The metric counts segments (closest-hit queries with their deposit and
shading) on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank traces its own copy of the workload (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
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
METRIC = "radio-map ray-bounces/s"
UNIT = "ray-bounces/s"
WORKLOAD = ("manhattan seed 2: 10x10 box buildings, 1202 triangles, 4 materials (ground half-space + 3 slab); "
            "1 TX at (0,0,30) m isotropic V-pol; 28 GHz; 1e7 Fibonacci rays; max depth 5 (R+T); "
            "512x512 map of 1 m cells at z=1.5 m")
PROFILE = os.path.join(ROOT, "profiles", "k_trace_manhattan_1e7.md")
# the tracer's code and the tree it walks (the LBVH build decides its node visits)
TRACE_SOURCES = [os.path.join(ROOT, "paper_2504_21719_b300", "csrc", f) for f in ("trace.cu", "common.cuh", "array.cuh", "bvh.cu")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rays", type=int, default=0, help="override the ray count (profiling a smaller case)")
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


def profiled(key: str):
    """A figure (dram_bytes_per_launch, issue_active_pct) of the tracer from the
    committed ncu summary, if the kernel source is unchanged since it was
    taken; else None."""
    try:
        txt = open(PROFILE).read()
    except OSError:
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


def tuned(gpu_name: str, key: str):
    from paper_2504_21719_b300.autotune import lookup
    return lookup(gpu_name, key)


def oracle_sample(target_s: float = 15.0, max_rays: int = 10_000_000):
    """The FP64 oracle, as it stands, on a bounded lattice subset of the workload."""
    import oracle
    from synth import scenes as S
    sc, txs, p = S.workload(2)
    tx = txs[0]

    def run(stride, begin=0):
        tx.ray_stride, tx.ray_begin = stride, begin
        t0 = time.perf_counter()
        r = oracle.radio_map(sc, tx, p, want_record=True)
        dt = time.perf_counter() - t0
        segs = int((r["record"][:, :, 0] != -2).sum())
        return segs, dt, tx.count()

    segs, dt, n = run(100)                        # calibration: 1e5 rays
    rate = n / max(dt, 1e-3)
    rays = int(min(max_rays, max(2e4, rate * target_s)))
    stride = max(1, tx.num_rays // rays)
    segs, dt, n = run(stride, 1)
    return {"value": segs / dt, "unit": "segments/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"workload lattice subset: 1 in {stride} of 1e7 rays ({n} rays, {segs} segments, "
                      f"{dt:.1f} s), FP64 brute force over 1202 triangles"}


# ----------------------------------------------------------------------------- our arm
def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2504_21719_b300 import api
    from synth import scenes as S

    gpu_name = torch.cuda.get_device_name(local)
    sc, txs, p = S.workload(2)
    tx = txs[0]
    if args.rays:
        tx.num_rays = args.rays
    blk, bps, qch, rfm = tuned(gpu_name, "manhattan")
    params = api.params_from(p, block_size=blk, blocks_per_sm=bps, queue_chunk=qch, refill_min=rfm)
    gs = api.Scene.from_obj(sc)
    maps = torch.empty((1, p.ny, p.nx), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # one step = the trace captured once as a CUDA graph (map clear, tracer, FP64 -> FP32
    # map) and replayed; the graph times its tracer node with events around it
    plan = api.TracePlan(gs, [tx], params, maps)
    for _ in range(args.warmup):
        plan.launch()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    # nvidia-smi needs a moment to start sampling: keep the GPU busy meanwhile
    t_end = time.perf_counter() + 0.6
    while time.perf_counter() < t_end:
        plan.launch()
    torch.cuda.synchronize()
    step_ms, kern_ms, segs, nodes, tris = [], [], [], [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()                         # L2 (126 MB) flushed between timed steps
        torch.cuda.synchronize()
        ev0.record()
        plan.launch()
        ev1.record()
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        st = plan.stats()
        kern_ms.append(st["kernel_ms"])
        segs.append(st["segments"])
        nodes.append(st["nodes_visited"])
        tris.append(st["tris_tested"])
    plan.free()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    total_segs = sum(segs)
    if dist:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        s = torch.tensor([total_segs], dtype=torch.float64, device="cuda")
        dist.all_reduce(s, op=dist.ReduceOp.SUM)
        total_ms, total_segs = float(t), float(s)
    value = total_segs / (total_ms / 1e3)

    # roofline of the tracer kernel (its launches timed with CUDA events on its stream)
    pk = peaks()
    peak = pk.get("hbm_gbs")
    kavg = statistics.mean(kern_ms) / 1e3
    seg_step = statistics.mean(segs)
    achieved = SEGMENT_BYTES * seg_step / kavg / 1e9
    traffic = profiled("dram_bytes_per_launch")
    issue = profiled("issue_active_pct")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak if peak else 6400.0,
                "unit": "GB/s", "frac": round(achieved / (peak if peak else 6400.0), 4),
                "traffic": traffic, "peak_source": "measured" if peak else "fallback",
                "algorithmic_bytes_per_segment": SEGMENT_BYTES,
                "kernel": "k_trace (persistent forward tracer)", "kernel_ms": round(1e3 * kavg, 4),
                "issue_slots_busy_frac": None if issue is None else round(issue / 100.0, 3),
                "binding_limit": "instruction issue (scene and maps stay in L1/L2; see profiles/)"}

    # end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        vh = torch.from_numpy(sc.verts).pin_memory()
        th = torch.from_numpy(sc.tris).pin_memory()
        mh = torch.from_numpy(sc.tri_mat).pin_memory()
        out_h = torch.empty((1, p.ny, p.nx), dtype=torch.float32).pin_memory()
        e_ms, e_segs = [], []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g2 = api.Scene(vh, th, mh, sc.mats)
            r = api.trace(g2, [tx], params, out=maps)
            out_h.copy_(maps, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            g2.free()
            if i >= args.warmup:
                e_ms.append(dt * 1e3)
                e_segs.append(r["stats"]["segments"])
        h2d = sc.verts.nbytes + sc.tris.nbytes + sc.tri_mat.nbytes + sc.mats.nbytes + 72 + 56
        e2e = {"value": sum(e_segs) / (sum(e_ms) / 1e3) * world, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(out_h.numel() * 4 + 576),
               "includes": "scene upload + LBVH build + trace + map readback, per step"}

    extra = {}
    if not args.no_extra and rank == 0:
        extra = run_extra(api, S, torch, gpu_name)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return None
    cpu = None
    if world == 1 and not args.no_cpu_baseline and not args.rays:
        cpu = oracle_sample()
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(statistics.mean(step_ms), 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays": tx.num_rays, "max_depth": p.max_depth, "map": [p.ny, p.nx],
                   "triangles": sc.nt, "segments_per_step": int(seg_step),
                   "nodes_per_segment": round(sum(nodes) / sum(segs), 2),
                   "tris_per_segment": round(sum(tris) / sum(segs), 2), "block_size": blk or 128,
                   "blocks_per_sm": bps or "max occupancy", "queue_chunk": qch or 1,
                   "refill_min": rfm or 20, "tuned": bool(blk),
                   "l2": "flushed between timed steps (256 MB write)",
                   "step": "CUDA graph of one trace (map clear, k_trace, k_map_to_f32), replayed",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps,
        "clocks": clk, "extra": extra,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return line


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


def run_extra(api, S, torch, gpu_name):
    """Batched 64-TX form, forward+adjoint of the differentiable workload, the
    large city, the widened model (diffuse reflection, early termination,
    synthetic arrays, diffraction, mesh surfaces) on the Manhattan workload, and
    the time-vs-N_S-and-N_A sweep on a street canyon."""
    import numpy as np

    out = {}
    # widened model on the 1e7-ray Manhattan workload (same scene, TX, map)
    sc, txs, p = S.workload(2)
    blk, bps, qch, rfm = tuned(gpu_name, "manhattan")
    kw = dict(block_size=blk, blocks_per_sm=bps, queue_chunk=qch, refill_min=rfm)
    base = _kernel_rate(api, api.Scene.from_obj(sc), txs, api.params_from(p, **kw))
    scd = sc.with_scattering(0.5, 0.2, np.arange(sc.nm) % 3, 3, 2, 0.6)
    pd = copy.copy(p)
    pd.diffuse = True
    gsd = api.Scene.from_obj(scd)
    d = _kernel_rate(api, gsd, txs, api.params_from(pd, **kw))
    d["vs_specular"] = round(d["value"] / base["value"], 3)
    d["materials"] = "S = 0.5 on every material; ground Lambertian, buildings directive / backscattering"
    out["specular_same_call"] = base
    out["diffuse"] = d
    gsd.free()
    pr = copy.copy(p)
    pr.rr_depth, pr.rr_max_prob = 2, 0.5
    gs = api.Scene.from_obj(sc)
    e = _kernel_rate(api, gs, txs, api.params_from(pr, **kw))
    e["setting"] = "Russian roulette after 2 interactions, p_max = 0.5"
    out["early_termination"] = e
    ta = copy.copy(txs[0])
    ta.ant_pos, ta.precoding = S.uniform_linear_array(64, p.freq_hz, 0.5, axis=0)
    a = _kernel_rate(api, gs, [ta], api.params_from(p, **kw))
    a["setting"] = "64-element half-wavelength ULA, uniform precoding"
    out["synthetic_array_64"] = a
    # first-order diffraction map of the same transmitter: 1200 wedges x 4096 samples
    wl = gs.wedges()
    for _ in range(2):
        api.diffraction_map(gs, txs, p, 4096, wedges=wl)
    dk, dst = [], None
    for _ in range(5):
        r = api.diffraction_map(gs, txs, p, 4096, wedges=wl)
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
    pm = api.params_from(p, **kw)
    for _ in range(2):
        api.trace_mesh(gs, su, txs, pm)
    mk, mst = [], None
    for _ in range(5):
        r = api.trace_mesh(gs, su, txs, pm)
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
    sc, txs, p = S.workload(3)
    blk, bps, qch, rfm = tuned(gpu_name, "batched")
    gs = api.Scene.from_obj(sc)
    prm = api.params_from(p, block_size=blk, blocks_per_sm=bps, queue_chunk=qch, refill_min=rfm)
    maps = torch.empty((len(txs), p.ny, p.nx), dtype=torch.float32, device="cuda")
    plan = api.TracePlan(gs, txs, prm, maps)
    for _ in range(3):
        plan.launch()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, segs = [], 0
    for _ in range(5):
        ev0.record()
        plan.launch()
        ev1.record()
        torch.cuda.synchronize()
        ms.append(ev0.elapsed_time(ev1))
        segs = plan.stats()["segments"]
    out["batched_64tx"] = {"value": round(segs / (statistics.mean(ms) / 1e3), 1), "unit": UNIT,
                           "ms_per_launch": round(statistics.mean(ms), 3), "segments": segs,
                           "rays": sum(t.num_rays for t in txs), "form": "CUDA graph, one persistent launch"}
    plan.free()
    gs.free()

    sc, txs, p = S.workload(4)
    gs = api.Scene.from_obj(sc)
    tgt_sc = S.Scene(sc.name, sc.verts, sc.tris, sc.tri_mat, S.perturb_materials(sc.mats, 40))
    gt = api.Scene.from_obj(tgt_sc)
    tgt = api.trace(gt, txs, p)["maps"][0]
    gt.free()
    f_ms, a_ms, b_ms, segs = [], [], [], 0
    for i in range(8):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = api.trace(gs, txs, p)
        loss, dL, _ = api.db_mse_loss(f["maps"][0], tgt)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        a = api.grad(gs, txs, p, dL.view(1, p.ny, p.nx))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if i >= 3:
            f_ms.append(f["stats"]["kernel_ms"])
            a_ms.append(a["stats"]["kernel_ms"])
            segs = f["stats"]["segments"]
            b_ms.append((t2 - t1) * 1e3)
    fk, ak = statistics.mean(f_ms), statistics.mean(a_ms)
    out["differentiable"] = {"fwd_kernel_ms": round(fk, 3), "adj_kernel_ms": round(ak, 3),
                             "fwd_plus_adj_over_fwd": round((fk + ak) / fk, 3),
                             "adj_call_ms": round(statistics.mean(b_ms), 3),
                             "fwd_plus_adj_call_over_fwd": round((fk + statistics.mean(b_ms)) / fk, 3),
                             "fwd_value": round(segs / (fk / 1e3), 1), "unit": UNIT}
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
    out["differentiable_diffuse"] = {"fwd_kernel_ms": round(statistics.mean(fk), 3),
                                     "adj_kernel_ms": round(statistics.mean(ak), 3),
                                     "fwd_plus_adj_over_fwd": round(1 + statistics.mean(ak) / statistics.mean(fk), 3)}
    gs.free()

    # large city: 0.97M triangles, 16 TX x 1e8 rays, depth 8, one launch each way
    sc, txs, p = S.workload(5)
    gs = api.Scene.from_obj(sc)
    blk, bps, qch, rfm = tuned(gpu_name, "city")
    p = api.params_from(p, block_size=blk, blocks_per_sm=bps, queue_chunk=qch, refill_min=rfm)
    small = [S.Tx(pos=txs[0].pos, num_rays=1_000_000, seed=txs[0].seed)]
    api.trace(gs, small, p)
    f = api.trace(gs, txs, p)
    g = torch.full_like(f["maps"], 1.0 / f["maps"].numel())
    a = api.grad(gs, txs, p, g)
    fk, ak = f["stats"]["kernel_ms"], a["stats"]["kernel_ms"]
    segs = f["stats"]["segments"]
    out["large_city"] = {"triangles": sc.nt, "rays": f["stats"]["rays"], "segments": segs,
                         "fwd_kernel_ms": round(fk, 1), "fwd_value": round(segs / (fk / 1e3), 1),
                         "adj_kernel_ms": round(ak, 1), "adj_value": round(segs / (ak / 1e3), 1),
                         "fwd_plus_adj_over_fwd": round((fk + ak) / fk, 3), "unit": UNIT,
                         "nodes_per_segment": round(f["stats"]["nodes_visited"] / segs, 2),
                         "tris_per_segment": round(f["stats"]["tris_tested"] / segs, 2)}
    del f, a, g
    gs.free()
    out["time_vs_samples_and_antennas"] = sweep_samples_antennas(api, S, torch, gpu_name)
    return out


def sweep_samples_antennas(api, S, torch, gpu_name, n_s=(10**6, 10**7, 10**8, 10**9), n_a=(1, 16, 128, 1024)):
    """Radio-map time of one transmitter 20 m above a street canyon as the number of
    samples N_S and of transmit-array elements N_A grow (the timing study of
    Sec. 4.5): depth 5, 3.5 GHz, 256 x 256 cells of 1 m, half-wavelength ULA with
    uniform precoding (N_A = 1: a single antenna).  Kernel time and the wall time
    of the `trace()` call, milliseconds, medians of two calls after one warm-up."""
    sc = S.street_canyon()
    gs = api.Scene.from_obj(sc)
    p = S.TraceParams(3.5e9, 5, cell_size=1.0, nx=256, ny=256)
    blk, bps, qch, rfm = tuned(gpu_name, "manhattan")
    prm = api.params_from(p, block_size=blk, blocks_per_sm=bps, queue_chunk=qch, refill_min=rfm)
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
    if rank != 0:
        return None
    import oracle
    from synth import scenes as S
    sc, txs, p = S.workload(2)
    tx = txs[0]
    stride = 50                                    # 2e5 rays per step
    times, segs = [], []
    for i in range(args.warmup + args.steps):
        tx.ray_stride, tx.ray_begin = stride, i % stride
        t0 = time.perf_counter()
        r = oracle.radio_map(sc, tx, p, want_record=True)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            segs.append(int((r["record"][:, :, 0] != -2).sum()))
    value = sum(segs) / sum(times)
    sample = (f"per step: 1 in {stride} rays of the 1e7-ray lattice ({tx.count()} rays), FP64 brute force over "
              f"{sc.nt} triangles, OpenMP")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(times), 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sampled": True},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
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
