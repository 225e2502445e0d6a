"""Pins of the CUDA path against physics rather than against the oracle's
replay: the two-ray closed form at N_S = 1e8, reciprocity at N_S = 1e8 per
replicate, and unbiasedness of the 1/Pr weighting (the mean of 64 seeds'
maps against the oracle's branch-all expectation)."""
import math

import numpy as np
import pytest
import torch

from synth import scenes as S
from closed_forms import (RECIP_A, RECIP_PAIRS, recip_params, recip_scene, reciprocity_bound,
                          reciprocity_replicates, two_ray)

pytestmark = pytest.mark.gpu


def test_two_ray_closed_form_1e8(api):
    """Workload 1 with 1e8 rays: every cell that n_i >= 100 rays cross (nearly
    the whole 200 m x 200 m map) is within 3 / sqrt(n_i) of the cell-averaged
    two-ray gain."""
    sc, txs, p = S.workload(1)
    tx = txs[0]
    tx.num_rays = 100_000_000
    gs = api.Scene.from_obj(sc)
    r = api.trace(gs, [tx], p)
    torch.cuda.synchronize()
    m = r["maps"][0].double().cpu().numpy()
    gs.free()
    assert r["stats"]["rays"] == tx.num_rays
    ref, n_i = two_ray(tx.pos, p, tx.num_rays)
    ok = n_i >= 100
    assert ok.sum() > 9000
    rel = np.abs(m / ref - 1)
    assert np.all(rel[ok] <= 3 / np.sqrt(n_i[ok])), rel[ok].max()


@pytest.mark.parametrize("deposit", [0, 1])
@pytest.mark.parametrize("rx", RECIP_PAIRS)
def test_reciprocity_1e8(api, rx, deposit):
    """The cell around B with the TX at A equals the cell around A with the TX
    at B (dual-polarised isotropic TX, ground + slab wall), each direction 16
    replicates of ~1e8 rays traced as one batched launch, 0.5 m cells."""
    sc, cell = recip_scene(), 0.5
    gs = api.Scene.from_obj(sc)
    vals = {}
    for tx_pos, rx_pos in ((RECIP_A, rx), (rx, RECIP_A)):
        txs = [S.Tx(pos=tx_pos, num_rays=n, pol=2, seed=seed)
               for n, seed in reciprocity_replicates(100_000_000, 16)]
        r = api.trace(gs, txs, recip_params(rx_pos, cell, deposit))
        torch.cuda.synchronize()
        vals[tx_pos] = r["maps"][:, 1, 1].double().cpu().numpy()
    gs.free()
    a, b = vals[RECIP_A], vals[rx]
    assert a.min() > 0 and b.min() > 0
    d = math.dist(RECIP_A, rx)
    assert abs(a.mean() - b.mean()) <= reciprocity_bound(a, b, cell, d), (a.mean(), b.mean(), a.std(), b.std())


def test_unbiased_mean_of_64_seeds_matches_branch_all(orc, api):
    """Importance sampling of the interaction type with 1/Pr weights
    (Eq. path-solver-used-dist-event, App. B) is unbiased: the mean of the GPU
    maps over 64 seeds (one batched launch) matches the oracle's branch-all
    expectation for the same lattice within 4.5 standard errors per cell.
    Cells reached only without a random choice have no spread; they must match
    to the per-cell parity tolerance of FP32 arithmetic (1e-3)."""
    sc = S.ground_and_wall(wall_mat=(4.0, 0.02, 0.2))
    N, L = 20_000, 3
    p = S.TraceParams(28e9, L, cell_size=4.0, nx=24, ny=24)
    pos = (0.0, 0.0, 10.0)
    exact, _, _ = orc.branch_all(sc, S.Tx(pos=pos, num_rays=N), p)
    gs = api.Scene.from_obj(sc)
    r = api.trace(gs, [S.Tx(pos=pos, num_rays=N, seed=s) for s in range(64)], p)
    torch.cuda.synchronize()
    maps = r["maps"].double().cpu().numpy()
    gs.free()
    mean, se = maps.mean(0), maps.std(0, ddof=1) / math.sqrt(len(maps))
    live = exact > 1e-15
    assert live.sum() > 400
    det = se <= 1e-6 * mean
    rnd = live & ~det
    assert rnd.sum() > 100
    assert np.all(np.abs(mean - exact)[rnd] <= 4.5 * se[rnd] + 1e-3 * exact[rnd])
    assert np.all(np.abs(mean - exact)[live & det] <= 1e-3 * exact[live & det])
    assert np.all(mean[~live] <= 1e-15)
