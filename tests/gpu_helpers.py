"""Shared helpers of the GPU parity tests (imported by tests only)."""
import numpy as np

MAP_RTOL = 1e-3          # per-cell relative tolerance of the maps
FLOOR = 1e-15            # cells above -150 dB are compared


def compare_maps(orc, scene, tx, params, gpu_map, gpu_record, rtol=MAP_RTOL, max_adopt_frac=5e-3):
    """Replay the GPU's discrete choices in the FP64 oracle (certifying every
    difference as a near-tie) and compare the maps cell by cell."""
    L = params.max_depth
    rec = np.asarray(gpu_record).reshape(tx.count(), L + 1, 4)
    r = orc.radio_map(scene, tx, params, mode="replay", record=rec)
    rep = r["report"]
    assert rep["failures"] == 0, rep
    adopted = rep["adopted_hit"] + rep["adopted_cell"] + rep["adopted_decision"]
    assert adopted <= max_adopt_frac * max(rep["segments"], 1) + 2, rep
    ref = r["map"]
    g = np.asarray(gpu_map, np.float64).reshape(ref.shape)
    mask = (ref > FLOOR) | (g > FLOOR)
    rel = np.abs(g - ref)[mask] / np.maximum(ref[mask], 1e-300)
    worst = float(rel.max()) if rel.size else 0.0
    assert worst <= rtol, (worst, int(mask.sum()), rep)
    assert np.all(g[~mask] <= FLOOR)
    return {"worst_rel": worst, "cells": int(mask.sum()), "report": rep}
