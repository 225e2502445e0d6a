"""Shared helpers of the GPU parity tests (imported by tests only)."""
import copy
import json
import os

import numpy as np

MAP_RTOL = 1e-3          # per-cell relative tolerance of the maps
FLOOR = 1e-15            # cells above -150 dB are compared
# Bilinear (tent) deposits: a weight is (1 - f) or f with f the FP32 fractional
# cell coordinate of the crossing x_c = o + t_c k.  FP32 origins carry errors
# |d o| <= eps (1 m + |o|_inf + path) and directions |d k| <= eps, which move
# the crossing by at most eps * D with
#   D = (1 + |o|_inf + path + t_c) (1 + (|k_x| + |k_y|) / |k_z|)
# (the oracle's conditioning factor: grazing rays that start near the plane,
# as diffuse reflections spawn them, are the ill-conditioned ones).  A tent
# weight w = w_x w_y then moves by at most 2 eps D / cell, so a cell may differ
# by 2 eps / cell times the D-weighted values of the deposits whose stencil
# covers it.  eps = 4 * 2^-24: a few FP32 roundings per coordinate.
POS_EPS = 4.0 * 2.0 ** -24
# Adopted near-ties, as fractions of the replayed segments.  Distance ties
# (the GPU's triangle is at the FP64 closest distance within tol: a box floor
# coplanar with the ground, resolved by index on both sides but with different
# tolerances) were measured at up to 0.8 % of segments (one transmitter of the
# batched workload), 0.33 % on the Manhattan subsets; every other adoption
# (hits that are not distance ties, cells, decisions) at up to 3e-5.  The caps
# are about 3x the measured maxima (plus a few for small replays).
MAX_ADOPT_FRAC = 2.5e-2          # distance-tie hit adoptions
MAX_OTHER_FRAC = 1e-4            # all other adoptions
MAX_DIFF_VIS_FRAC = 1e-3         # diffraction visibility bits (measured 2.9e-4)
# The GPU's recorded coin probabilities (RM_RECORD_COIN) were measured within
# 0.26 of the replay's decision window of the oracle's q(R) on every parity
# workload (6e-5 at most, city depth 8); they must stay within half of it.
MAX_COIN_RATIO = 0.5


def _log(kind, rep, extra=None):
    """Append one replay report to the file named by RM_PARITY_LOG (if set), so
    that a GPU run can collect the adoption rates of every parity test."""
    path = os.environ.get("RM_PARITY_LOG")
    if not path:
        return
    test = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    row = {"test": test, "kind": kind, **{k: v for k, v in rep.items() if k != "fail_info"}}
    if extra:
        row.update(extra)
    with open(path, "a") as f:
        f.write(json.dumps(row) + "\n")


def coin(params):
    """A copy of the trace parameters whose debug record also carries the
    GPU's coin probability q(R) of every decision (RM_RECORD_COIN)."""
    q = copy.copy(params)
    q.record_coin = True
    return q


def check_coins(rep):
    """When the GPU recorded its coin probabilities (RM_RECORD_COIN), every one
    must lie inside half of the replay's decision window around the oracle's q(R)."""
    if rep.get("coin_checked", 0) > 0:
        assert rep["coin_outside"] == 0, rep
        assert rep["coin_max_ratio"] <= MAX_COIN_RATIO, rep


def check_adoptions(rep, max_adopt_frac=MAX_ADOPT_FRAC, max_other_frac=MAX_OTHER_FRAC):
    """Distance-tie hit adoptions and all other adoptions, each under its cap."""
    seg = max(rep["segments"], 1)
    ties = rep.get("adopted_hit_tie", 0)
    other = rep["adopted_hit"] - ties + rep.get("adopted_cell", 0) + rep["adopted_decision"]
    assert ties <= max_adopt_frac * seg + 2, rep
    assert other <= max_other_frac * seg + 3, rep


def compare_maps(orc, scene, tx, params, gpu_map, gpu_record, rtol=MAP_RTOL, max_adopt_frac=MAX_ADOPT_FRAC):
    """Replay the GPU's discrete choices in the FP64 oracle (certifying every
    difference as a near-tie) and compare the maps cell by cell."""
    L = params.max_depth
    rec = np.asarray(gpu_record).reshape(tx.count(), L + 1, 4)
    bil = params.deposit == 1
    arr = getattr(tx, "ant_pos", None) is not None and len(tx.ant_pos) > 0
    r = orc.radio_map(scene, tx, params, mode="replay", record=rec, mass=bil or arr)
    rep = r["report"]
    _log("map", rep)
    assert rep["failures"] == 0, rep
    check_coins(rep)
    check_adoptions(rep, max_adopt_frac)
    ref = r["map"]
    g = np.asarray(gpu_map, np.float64).reshape(ref.shape)
    mask = (ref > FLOOR) | (g > FLOOR)
    err = np.abs(g - ref)[mask]
    bound = rtol * ref[mask]
    if bil:
        bound = bound + 2.0 * POS_EPS / params.cell_size * r["cmass"][mask]
    if arr:
        # FP32 array factor: first-order propagation of the kernel's direction
        # and phase roundings through |alpha|^2 (the oracle's array conditioning)
        bound = bound + r["amass"][mask]
    rel = err / np.maximum(ref[mask], 1e-300)
    worst = float((err / np.maximum(bound, 1e-300)).max()) if err.size else 0.0
    assert np.all(err <= bound), (worst, float(rel.max()), int(mask.sum()), rep)
    assert np.all(g[~mask] <= FLOOR)
    out = {"worst_rel": float(rel.max()) if rel.size else 0.0, "worst_vs_bound": worst,
           "cells": int(mask.sum()), "report": rep}
    if arr:
        # the array bound is a worst case; report how many cells meet the plain tolerance
        out["frac_within_rtol"] = float(np.mean(err <= rtol * ref[mask])) if err.size else 1.0
    return out


def compare_diffraction(orc, scene, tx, params, samples_per_wedge, gpu_map, gpu_record, rtol=MAP_RTOL,
                        max_adopt_frac=MAX_ADOPT_FRAC, wedge_index=None):
    """Replay the GPU's visibility bits and cells of a diffraction map in the
    FP64 oracle (every difference certified as a near-tie), then compare the
    maps cell by cell.  wedge_index: the GPU sampled only these wedges (positions
    in the oracle's wedge list), in this order."""
    rec = np.asarray(gpu_record).reshape(-1, 4)
    r = orc.diffraction_map(scene, tx, params, samples_per_wedge, mode="replay", record=rec, slack=True,
                            wedge_index=wedge_index)
    rep = r["report"]
    _log("diffraction", rep)
    assert rep["failures"] == 0, rep
    seg = max(rep["segments"], 1)
    assert rep["adopted_hit"] <= MAX_DIFF_VIS_FRAC * seg + 2, rep
    assert rep["adopted_cell"] + rep["adopted_decision"] <= MAX_OTHER_FRAC * seg + 3, rep
    ref = r["map"]
    g = np.asarray(gpu_map, np.float64).reshape(ref.shape)
    mask = (ref > FLOOR) | (g > FLOOR)
    err = np.abs(g - ref)[mask]
    # the UTD field jumps across shadow boundaries (and where N^+- rounds the
    # other way): FP32 angles, good to ~1e-6 rad, may put a sample on the other
    # side of one; the oracle reports per cell how much its deposits change under
    # a +-1e-5 rad shift of the Keller azimuth, which bounds such flips
    bound = rtol * ref[mask] + r["slack"][mask]
    rel = err / np.maximum(ref[mask], 1e-300)
    worst = float((err / np.maximum(bound, 1e-300)).max()) if err.size else 0.0
    assert np.all(err <= bound), (worst, float(rel.max()), int(mask.sum()), rep)
    assert np.all(g[~mask] <= FLOOR)
    return {"worst_rel": float(rel.max()) if rel.size else 0.0, "cells": int(mask.sum()), "report": rep}


def compare_mesh(orc, scene, tx, params, surf_v, surf_t, gpu_map, gpu_record, rtol=MAP_RTOL,
                 max_adopt_frac=MAX_ADOPT_FRAC):
    """Replay the GPU's hits and decisions in the FP64 oracle on a mesh
    measurement surface and compare cell by cell.  A crossing within tol of a
    triangle's boundary (or of the segment's window) may land on either side in
    FP32; the oracle's per-cell slack bounds those."""
    L = params.max_depth
    rec = np.asarray(gpu_record).reshape(tx.count(), L + 1, 4)
    r = orc.radio_map_mesh(scene, tx, params, surf_v, surf_t, mode="replay", record=rec, slack=True)
    rep = r["report"]
    _log("mesh", rep)
    assert rep["failures"] == 0, rep
    check_coins(rep)
    check_adoptions(rep, max_adopt_frac)
    ref = r["map"]
    g = np.asarray(gpu_map, np.float64).reshape(ref.shape)
    mask = (ref > FLOOR) | (g > FLOOR)
    err = np.abs(g - ref)[mask]
    bound = rtol * ref[mask] + r["slack"][mask]
    rel = err / np.maximum(ref[mask], 1e-300)
    worst = float((err / np.maximum(bound, 1e-300)).max()) if err.size else 0.0
    assert np.all(err <= bound), (worst, float(rel.max()), int(mask.sum()), rep)
    assert np.all(g[~mask] <= FLOOR)
    return {"worst_rel": float(rel.max()) if rel.size else 0.0, "cells": int(mask.sum()), "report": rep}


def compare_diffraction_mesh(orc, scene, tx, params, samples_per_wedge, surf_v, surf_t, gpu_map, gpu_record,
                             rtol=MAP_RTOL, max_adopt_frac=MAX_ADOPT_FRAC, wedge_index=None):
    """Replay the GPU's incident-visibility bits in the FP64 oracle's diffraction
    map on a mesh surface and compare cell by cell.  Crossings near a triangle's
    boundary, visibility near ties of the edge-to-crossing segments and a
    +-1e-5 rad Keller azimuth change are bounded by the oracle's per-cell slack."""
    rec = np.asarray(gpu_record).reshape(-1, 4)
    r = orc.diffraction_map_mesh(scene, tx, params, samples_per_wedge, surf_v, surf_t, mode="replay", record=rec,
                                 slack=True, wedge_index=wedge_index)
    rep = r["report"]
    _log("diffraction_mesh", rep)
    assert rep["failures"] == 0, rep
    assert rep["adopted_hit"] <= MAX_DIFF_VIS_FRAC * max(rep["segments"], 1) + 2, rep
    ref = r["map"]
    g = np.asarray(gpu_map, np.float64).reshape(ref.shape)
    mask = (ref > FLOOR) | (g > FLOOR)
    err = np.abs(g - ref)[mask]
    bound = rtol * ref[mask] + r["slack"][mask]
    rel = err / np.maximum(ref[mask], 1e-300)
    worst = float((err / np.maximum(bound, 1e-300)).max()) if err.size else 0.0
    assert np.all(err <= bound), (worst, float(rel.max()), int(mask.sum()), rep)
    assert np.all(g[~mask] <= FLOOR)
    return {"worst_rel": float(rel.max()) if rel.size else 0.0, "cells": int(mask.sum()), "report": rep}
