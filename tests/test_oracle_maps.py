"""Pins of the oracle's radio-map estimator (Eq. radio-map-solver-ci-all-2-estimator)
against closed forms (Friis, two-ray), exact energy bookkeeping, unbiasedness,
and of its replay / frozen / gradient modes (CPU only)."""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

from synth import scenes as S
from closed_forms import (C0, RECIP_A, RECIP_PAIRS, cell_avg as _cell_avg, recip_params, recip_scene,
                          reciprocity_bound, reciprocity_replicates, two_ray)

# ---------------------------------------------------------------------------
# one ray -> one deposit, exactly the estimator's term
# ---------------------------------------------------------------------------
def test_single_ray_deposit_closed_form(orc):
    sc = S.empty_scene()
    f, cell = 3.5e9, 2.0
    lam = C0 / f
    # N = 2: ray 1 points straight down (pole); |E|^2 = 1, |k_z| = 1
    tx = S.Tx(pos=(3.3, -2.2, 10.0), num_rays=2, ray_begin=1, ray_count=1)
    p = S.TraceParams(f, 0, cell_size=cell, nx=10, ny=10)
    m = orc.radio_map(sc, tx, p)["map"]
    want = 4 * math.pi / (2 * cell * cell) * (lam / (4 * math.pi)) ** 2
    iy, ix = int((-2.2 + 10) // cell), int((3.3 + 10) // cell)
    assert abs(m[iy, ix] - want) <= 1e-12 * want and np.count_nonzero(m) == 1
    # a slanted lattice ray: direction from the lattice definition at 50 digits
    getcontext().prec = 50
    N, n = 1000, 801
    z = 1 - 2 * n / (N - 1)
    q = Decimal(n) / ((1 + Decimal(5).sqrt()) / 2)
    ph = 2 * math.pi * float(q - int(q))
    st = math.sqrt(1 - z * z)
    k = np.array([st * math.cos(ph), st * math.sin(ph), z])
    tx = S.Tx(pos=(0.0, 0.0, 10.0), num_rays=N, ray_begin=n, ray_count=1)
    p = S.TraceParams(f, 0, cell_size=cell, nx=40, ny=40)
    m = orc.radio_map(sc, tx, p)["map"]
    t = (1.5 - 10.0) / k[2]
    x, y = t * k[0], t * k[1]
    want = 4 * math.pi / (N * cell * cell) * (lam / (4 * math.pi)) ** 2 / abs(k[2])
    iy, ix = int((y + 40) // cell), int((x + 40) // cell)
    assert abs(m[iy, ix] - want) <= 1e-12 * want and np.count_nonzero(m) == 1


def test_upward_ray_and_parallel_ray_do_not_deposit(orc):
    sc = S.empty_scene()
    p = S.TraceParams(1e9, 0, cell_size=1.0, nx=8, ny=8)
    up = S.Tx(pos=(0.0, 0.0, 10.0), num_rays=2, ray_begin=0, ray_count=1)   # +z, above plane
    horiz = S.Tx(pos=(0.0, 0.0, 1.5), num_rays=1)                           # N = 1: horizontal
    assert orc.radio_map(sc, up, p)["map"].sum() == 0.0
    assert orc.radio_map(sc, horiz, p)["map"].sum() == 0.0


# ---------------------------------------------------------------------------
# free space: cell average of Friis' (lambda / 4 pi d)^2
# ---------------------------------------------------------------------------
def test_free_space_matches_friis(orc):
    sc = S.empty_scene()
    f, h, zm, cell, nx = 3.5e9, 10.0, 1.5, 2.0, 20
    lam = C0 / f
    N = 1_000_000
    tx = S.Tx(pos=(0.0, 0.0, h), num_rays=N)
    p = S.TraceParams(f, 0, cell_size=cell, nx=nx, ny=nx, map_origin=(0, 0, zm))
    m = orc.radio_map(sc, tx, p)["map"]
    x0 = -nx * cell / 2
    ref = _cell_avg(lambda X, Y: (lam / (4 * math.pi)) ** 2 / (X ** 2 + Y ** 2 + (h - zm) ** 2),
                    x0, x0, cell, nx, nx)
    # expected number of rays through each cell (tube density times area)
    n_i = _cell_avg(lambda X, Y: N / (4 * math.pi) * (h - zm) / (X ** 2 + Y ** 2 + (h - zm) ** 2) ** 1.5,
                    x0, x0, cell, nx, nx) * cell * cell
    rel = np.abs(m / ref - 1)
    ok = n_i >= 100
    assert ok.sum() > 300
    assert np.all(rel[ok] <= 3 / np.sqrt(n_i[ok])), rel[ok].max()
    # the map integrates the gain over the plane: sum * cell^2 = power through the window
    assert abs((m * ref > 0).mean() - 1) < 1e-12


# ---------------------------------------------------------------------------
# two-ray model over the ground half-space (workload 1, V-pol is pure TM)
# ---------------------------------------------------------------------------
def test_two_ray_ground_plane(orc):
    """Workload 1 at N_S = 1e7 rays against the cell-averaged two-ray gain,
    within 3 / sqrt(n_i) for every cell that n_i >= 100 rays cross."""
    sc, txs, p = S.workload(1)
    tx = txs[0]
    tx.num_rays = 10_000_000
    m = orc.radio_map(sc, tx, p)["map"]
    ref, n_i = two_ray(tx.pos, p, tx.num_rays)
    rel = np.abs(m / ref - 1)
    ok = n_i >= 100
    assert ok.sum() > 4000
    assert np.all(rel[ok] <= 3 / np.sqrt(n_i[ok])), rel[ok].max()


# ---------------------------------------------------------------------------
# reciprocity: ground + one slab wall, dual-polarised isotropic TX
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("deposit", [0, 1])
@pytest.mark.parametrize("rx", RECIP_PAIRS)
def test_reciprocity_ground_and_wall(orc, rx, deposit):
    """The centre cell around B with the TX at A equals the centre cell around
    A with the TX at B.  Reciprocity of the propagation (App. A.5: Fresnel and
    slab coefficients depend only on the incidence angle; the spreading of
    specular paths is symmetric) makes the transfer matrix of the reversed path
    the transpose of the forward one in the theta/phi bases (up to the sign of
    phi-hat), so its Frobenius norm is reciprocal.  A dual-polarised isotropic
    TX maps exactly that norm (the sum of both columns' |T C|^2, Sec. 4.4),
    while a single V column is not polarisation-pure once ground-then-wall
    paths mix it.  16 replicates of ~1e6 rays in each direction."""
    sc, cell = recip_scene(), 1.0
    vals = {}
    for tx_pos, rx_pos in ((RECIP_A, rx), (rx, RECIP_A)):
        v = []
        for n, seed in reciprocity_replicates(1_000_000, 16):
            t = S.Tx(pos=tx_pos, num_rays=n, pol=2, seed=seed)
            v.append(orc.radio_map(sc, t, recip_params(rx_pos, cell, deposit))["map"][1, 1])
        vals[tx_pos] = np.array(v)
    a, b = vals[RECIP_A], vals[rx]
    d = math.dist(RECIP_A, rx)
    assert a.min() > 0 and b.min() > 0
    assert abs(a.mean() - b.mean()) <= reciprocity_bound(a, b, cell, d), (a.mean(), b.mean())


# ---------------------------------------------------------------------------
# energy bookkeeping: branch-all on a closed lossless box
# ---------------------------------------------------------------------------
def test_branch_all_energy_lossless_closed_box(orc):
    sc = S.closed_box(10.0, mat=(3.0, 0.0, 0.2))
    N, L = 300, 6
    tx = S.Tx(pos=(1.0, 2.0, 3.0), num_rays=N)
    p = S.TraceParams(28e9, L, cell_size=1.0, nx=20, ny=20, map_origin=(0, 0, -2.0))
    _, pw, esc = orc.branch_all(sc, tx, p)
    # every interaction splits power exactly into R + T (|r|^2 + |t|^2 = 1):
    # power alive at segment l plus everything that escaped before = N
    for l in range(L + 1):
        tot = pw[l] + esc[:l].sum()
        assert abs(tot - N) <= 1e-12 * N, (l, tot)
    assert esc[0] == 0.0 and esc[2] > 0  # first escapes after one transmission


def test_branch_all_lossy_power_decreases(orc):
    sc, _, _ = S.workload(2)
    N, L = 200, 4
    tx = S.Tx(pos=(0.0, 0.0, 30.0), num_rays=N)
    p = S.TraceParams(28e9, L, cell_size=2.0, nx=64, ny=64)
    _, pw, esc = orc.branch_all(sc, tx, p)
    alive = pw - esc
    assert np.all(np.diff(pw) <= 1e-12 * N)
    assert np.all(pw[1:] <= alive[:-1] * (1 + 1e-12))


# ---------------------------------------------------------------------------
# unbiasedness: mean of MC maps over seeds -> branch-all expectation
# ---------------------------------------------------------------------------
def test_mc_mean_matches_branch_all(orc):
    sc = S.ground_and_wall(wall_mat=(4.0, 0.02, 0.2))
    N, L = 3000, 3
    p = S.TraceParams(28e9, L, cell_size=4.0, nx=24, ny=24)
    exact, pw_exact, _ = orc.branch_all(sc, S.Tx(pos=(0.0, 0.0, 10.0), num_rays=N), p)
    maps, pws = [], []
    for seed in range(48):
        r = orc.radio_map(sc, S.Tx(pos=(0.0, 0.0, 10.0), num_rays=N, seed=seed), p, stats=True)
        maps.append(r["map"])
        pws.append(r["power"])
    maps, pws = np.array(maps), np.array(pws)
    mean, se = maps.mean(0), maps.std(0, ddof=1) / math.sqrt(len(maps))
    det = se == 0
    assert np.all(np.abs(mean - exact)[~det] <= 4.5 * se[~det] + 1e-9 * exact[~det])
    assert np.all(np.abs(mean - exact)[det] <= 1e-9 * exact[det])
    pm, ps = pws.mean(0), pws.std(0, ddof=1) / math.sqrt(len(pws))
    assert np.all(np.abs(pm - pw_exact) <= 4.5 * ps + 1e-9 * pw_exact)


# ---------------------------------------------------------------------------
# replay / frozen modes
# ---------------------------------------------------------------------------
def _small_manhattan():
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride, tx.ray_count = 997, 10000
    p.nx = p.ny = 256
    p.cell_size = 2.0
    return sc, tx, p


def test_replay_of_own_record_is_exact(orc):
    sc, tx, p = _small_manhattan()
    a = orc.radio_map(sc, tx, p, want_record=True)
    b = orc.radio_map(sc, tx, p, mode="replay", record=a["record"])
    rep = b["report"]
    assert rep["failures"] == 0 and rep["adopted_hit"] == rep["adopted_cell"] == rep["adopted_decision"] == 0
    assert np.array_equal(a["map"], b["map"])
    c = orc.radio_map(sc, tx, p, mode="frozen", record=a["record"])
    assert np.array_equal(a["map"], c["map"])


def test_replay_rejects_planted_mismatches(orc):
    sc, tx, p = _small_manhattan()
    a = orc.radio_map(sc, tx, p, want_record=True)
    rec = a["record"]
    # (1) a hit replaced by a far-away building triangle
    hit = np.argwhere(rec[:, 1, 0] >= 2)[0, 0]
    r1 = rec.copy()
    r1[hit, 1, 0] = 2 if rec[hit, 1, 0] > 600 else 1200
    assert orc.radio_map(sc, tx, p, mode="replay", record=r1)["report"]["fail_kind"] == 1
    # (2) a deposit moved by three cells
    dep = np.argwhere(rec[:, 0, 1] != orc.NO_CELL)[0, 0]
    r2 = rec.copy()
    r2[dep, 0, 1] = (r2[dep, 0, 1] + 3) % p.nx
    assert orc.radio_map(sc, tx, p, mode="replay", record=r2)["report"]["fail_kind"] == 2
    # (3) a flipped reflection / refraction decision (far from a tie)
    cand = np.argwhere((rec[:, 0, 3] >= 0) & (rec[:, 0, 0] >= 2))
    r3 = rec.copy()
    i = cand[len(cand) // 2, 0]
    r3[i, 0, 3] = 1 - r3[i, 0, 3]
    rep = orc.radio_map(sc, tx, p, mode="replay", record=r3)["report"]
    assert rep["fail_kind"] == 3 or (rep["failures"] == 0 and rep["adopted_decision"] == 1)


# ---------------------------------------------------------------------------
# gradient: dual numbers vs central finite differences, both with frozen choices
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("deposit", [1, 0])
def test_grad_dual_matches_frozen_fd(orc, deposit):
    sc, txs, p = S.workload(4)
    tx = txs[0]
    tx.ray_stride, tx.ray_count = 331, 3000
    p.deposit = deposit
    p.nx = p.ny = 96
    base = orc.radio_map(sc, tx, p, want_record=True)
    rec = base["record"]
    rng = np.random.default_rng(11)
    g = rng.normal(size=(p.ny, p.nx))
    d_eps, d_sig, d_tx = orc.grad(sc, tx, p, rec, g)
    mats0 = sc.mats.astype(np.float64)[:, :2]
    nm = len(mats0)

    def J(mats=mats0, pos=tx.pos):
        t = S.Tx(**{**tx.__dict__, "pos": tuple(pos)})
        return (orc.radio_map(sc, t, p, mode="frozen", record=rec, sampling_mats=mats0,
                              eval_mats=mats)["map"] * g).sum()

    fd = []
    for j in range(2 * nm):
        m, c = j % nm, j // nm
        # the slab phase turns by ~50 rad per unit permittivity at 28 GHz, so
        # the step must be small for O(h^2) truncation to stay below 1e-6
        h = 1e-6 * abs(mats0[m, c])
        mp, mm = mats0.copy(), mats0.copy()
        mp[m, c] += h
        mm[m, c] -= h
        fd.append((J(mats=mp) - J(mats=mm)) / (2 * h))
    for a in range(3):
        h = 1e-5 * max(abs(tx.pos[a]), 1.0)
        pp, pm = list(tx.pos), list(tx.pos)
        pp[a] += h
        pm[a] -= h
        fd.append((J(pos=pp) - J(pos=pm)) / (2 * h))
    fd = np.array(fd)
    ad = np.concatenate([d_eps, d_sig, d_tx])
    scale = np.maximum(np.abs(ad), 1e-3 * np.abs(ad).max())
    assert np.all(np.abs(ad - fd) <= 1e-6 * scale), np.abs(ad - fd) / scale
    if deposit == 0:
        # box cells: with frozen cells the map does not depend on the TX position
        assert np.all(d_tx == 0.0)
    else:
        assert np.abs(d_tx).max() > 0
