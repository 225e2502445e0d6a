"""GPU parity of the 'next' rows: synthetic transmit arrays (Sec. 4.5) and
early termination by gain thresholding and Russian roulette (Sec. 4.7)."""
import copy

import numpy as np
import pytest
import torch

from synth import scenes as S
from gpu_helpers import compare_maps

pytestmark = pytest.mark.gpu


def _manhattan(stride=97):
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = stride
    return sc, tx, p


def _run(api, sc, tx, p):
    gs = api.Scene.from_obj(sc)
    r = api.trace(gs, [tx], p, record=True)
    torch.cuda.synchronize()
    out = (r["maps"][0].cpu().numpy(), r["record"].cpu().numpy(), r["stats"])
    gs.free()
    return out


@pytest.mark.parametrize("nant,steer", [(8, (1.0, 0.2, -0.3)), (32, None)])
def test_synthetic_array(orc, api, nant, steer):
    sc, tx, p = _manhattan()
    tx.ant_pos, tx.precoding = S.uniform_linear_array(nant, p.freq_hz, 0.5, axis=0, steer=steer)
    tx.yaw = 0.4
    m, rec, _ = _run(api, sc, tx, p)
    compare_maps(orc, sc, tx, p, m, rec)


@pytest.mark.parametrize("rr_depth,pmax,thr", [(2, 0.0, 1e-12), (1, 0.3, 0.0), (2, 0.5, 3e-13)])
def test_early_termination(orc, api, rr_depth, pmax, thr):
    sc, tx, p = _manhattan()
    p.rr_depth, p.rr_max_prob, p.gain_threshold = rr_depth, pmax, thr
    m, rec, st = _run(api, sc, tx, p)
    dec = rec[:, 3]
    kills = int(((dec >= 0) & ((dec & 12) != 0)).sum())
    assert kills > 0
    compare_maps(orc, sc, tx, p, m, rec)
    # fewer segments than without early termination
    p0 = copy.copy(p)
    p0.rr_depth = 0
    _, _, st0 = _run(api, sc, tx, p0)
    assert st["segments"] < st0["segments"]


def test_adjoint_retakes_roulette_and_array(api):
    sc, txs, p = S.workload(4)
    tx = txs[0]
    tx.ray_stride = 13
    tx.ant_pos, tx.precoding = S.uniform_linear_array(4, p.freq_hz, 0.5, axis=1)
    p.rr_depth, p.rr_max_prob = 1, 0.4
    gs = api.Scene.from_obj(sc)
    f = api.trace(gs, [tx], p, record=True)
    a = api.grad(gs, [tx], p, torch.rand_like(f["maps"]), record=True)
    assert torch.equal(f["record"], a["record"])
    gs.free()
