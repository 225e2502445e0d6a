"""Pins of the oracle's synthetic transmit arrays (Sec. 4.4, Eq.
path-solver-array-response-vector) and early termination (Sec. 4.5, Eq.
radio-map-solver-rr-prob)."""
import copy
import math
from decimal import Decimal, getcontext

import numpy as np

from synth import scenes as S

C0 = 299792458.0


def test_single_element_array_is_identity(orc):
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 4999
    a = orc.radio_map(sc, tx, p)["map"]
    t1 = copy.copy(tx)
    t1.ant_pos, t1.precoding = np.zeros((1, 3)), np.array([1.0 + 0j])
    b = orc.radio_map(sc, t1, p)["map"]
    assert np.array_equal(a, b)


def test_two_element_array_single_ray_closed_form(orc):
    f, cell = 3.5e9, 2.0
    lam = C0 / f
    getcontext().prec = 50
    N, n = 1000, 801
    z = 1 - 2 * n / (N - 1)
    q = Decimal(n) / ((1 + Decimal(5).sqrt()) / 2)
    ph = 2 * math.pi * float(q - int(q))
    st = math.sqrt(1 - z * z)
    k = np.array([st * math.cos(ph), st * math.sin(ph), z])
    pos, w = S.uniform_linear_array(2, f, 0.5, axis=1)          # +-lambda/4 on y, weights 1/sqrt(2)
    tx = S.Tx(pos=(0.0, 0.0, 10.0), num_rays=N, ray_begin=n, ray_count=1, ant_pos=pos, precoding=w)
    p = S.TraceParams(f, 0, cell_size=cell, nx=40, ny=40)
    m = orc.radio_map(S.empty_scene(), tx, p)["map"]
    base = 4 * math.pi / (N * cell * cell) * (lam / (4 * math.pi)) ** 2 / abs(k[2])
    af = 2 * math.cos(math.pi * k[1] / 2) ** 2                 # |e^{j pi ky/2} + e^{-j pi ky/2}|^2 / 2
    assert abs(m.sum() - base * af) <= 1e-12 * base * af and np.count_nonzero(m) == 1


def test_half_wavelength_array_radiates_precoding_norm(orc):
    # With lambda/2 spacing the cross terms of |alpha|^2 integrate to
    # sinc(pi m) = 0, so the power through the sphere is 4 pi |u_P|^2.
    f = 28e9
    N = 200_000
    for nant, steer in ((4, None), (8, (1.0, 0.3, -0.2))):
        pos, w = S.uniform_linear_array(nant, f, 0.5, axis=0, steer=steer)
        tx = S.Tx(pos=(0.0, 0.0, 10.0), num_rays=N, ant_pos=pos, precoding=w, yaw=0.3, pitch=0.2)
        p = S.TraceParams(f, 0, cell_size=1.0, nx=4, ny=4)
        st = orc.radio_map(S.empty_scene(), tx, p, stats=True)
        mean_af = st["power"][0] / N                          # isotropic element: |E0|^2 = 1
        assert abs(mean_af - np.vdot(w, w).real) < 2e-3, mean_af


def _rr_params(L=4, rr_depth=1, pmax=0.5, thr=0.0):
    return S.TraceParams(28e9, L, cell_size=4.0, nx=24, ny=24, rr_depth=rr_depth, rr_max_prob=pmax,
                         gain_threshold=thr)


def test_russian_roulette_is_unbiased(orc):
    """Roulette keeps the expectation (branch-all without roulette) of the
    total map and of the power per depth.  Per-cell tests do not apply: cells
    fed by rare survivors of weight 1/p have heavy-tailed values."""
    sc = S.ground_and_wall(wall_mat=(4.0, 0.02, 0.2))
    N = 3000
    p = _rr_params()
    exact, pw_exact, _ = orc.branch_all(sc, S.Tx(pos=(0.0, 0.0, 10.0), num_rays=N), p)
    tot, pws, segs = [], [], []
    for seed in range(64):
        r = orc.radio_map(sc, S.Tx(pos=(0.0, 0.0, 10.0), num_rays=N, seed=seed), p, want_record=True,
                          stats=True)
        tot.append(r["map"].sum())
        pws.append(r["power"])
        segs.append(int((r["record"][:, :, 0] != -2).sum()))
    tot, pws = np.array(tot), np.array(pws)
    assert abs(tot.mean() - exact.sum()) <= 4.5 * tot.std(ddof=1) / math.sqrt(len(tot))
    pm, ps = pws.mean(0), pws.std(0, ddof=1) / math.sqrt(len(pws))
    assert np.all(np.abs(pm - pw_exact) <= 4.5 * ps + 1e-9 * pw_exact), (pm, pw_exact, ps)
    plain = orc.radio_map(sc, S.Tx(pos=(0.0, 0.0, 10.0), num_rays=N, seed=0), _rr_params(pmax=0.0),
                          want_record=True)
    assert np.mean(segs) < int((plain["record"][:, :, 0] != -2).sum())   # roulette stops paths


def test_gain_threshold_only_removes_power_and_replays(orc):
    sc, txs, p0 = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 997
    p0.nx = p0.ny = 128
    p0.cell_size = 4.0
    a = orc.radio_map(sc, tx, p0, want_record=True)
    p = copy.copy(p0)
    p.rr_depth, p.gain_threshold = 2, 1e-11
    b = orc.radio_map(sc, tx, p, want_record=True)
    assert np.all(b["map"] <= a["map"] * (1 + 1e-12)) and b["map"].sum() < a["map"].sum()
    killed = (b["record"][:, :, 3] >= 0) & ((b["record"][:, :, 3] & 8) != 0)
    assert killed.sum() > 0
    # replay of its own record is exact; a planted kill bit is rejected
    r = orc.radio_map(sc, tx, p, mode="replay", record=b["record"])
    assert r["report"]["failures"] == 0 and np.array_equal(r["map"], b["map"])
    rec = b["record"].copy()
    i, l = np.argwhere(killed)[0]
    rec[i, l, 3] &= ~8
    assert orc.radio_map(sc, tx, p, mode="replay", record=rec)["report"]["failures"] == 1


def test_roulette_replay_and_planted_kill(orc):
    sc, txs, p0 = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 997
    p = copy.copy(p0)
    p.nx = p.ny = 128
    p.cell_size = 4.0
    p.rr_depth, p.rr_max_prob = 1, 0.3
    b = orc.radio_map(sc, tx, p, want_record=True)
    rec = b["record"]
    r = orc.radio_map(sc, tx, p, mode="replay", record=rec)
    assert r["report"]["failures"] == 0 and np.array_equal(r["map"], b["map"])
    alive = np.argwhere((rec[:, :, 3] >= 0) & ((rec[:, :, 3] & 4) == 0) & (rec[:, :, 0] >= 0))
    bad = rec.copy()
    i, l = alive[len(alive) // 2]
    bad[i, l, 3] |= 4
    rep = orc.radio_map(sc, tx, p, mode="replay", record=bad)["report"]
    assert rep["failures"] >= 1
