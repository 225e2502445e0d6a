"""Adjoint kernel vs the oracle's dual-number gradient (same frozen choices,
taken from the GPU's own record) and vs GPU finite differences; dB loss."""
import copy
import math

import numpy as np
import pytest
import torch

from synth import scenes as S
from gpu_helpers import compare_maps

pytestmark = pytest.mark.gpu
GRAD_RTOL = 1e-2


def _setup(stride=13, deposit=1):
    sc, txs, p = S.workload(4)
    tx = txs[0]
    tx.ray_stride = stride
    p.deposit = deposit
    p.record_coin = True              # records carry the GPU's coin probabilities
    return sc, tx, p


def _target(api, sc, tx, p):
    tgt = S.perturb_materials(sc.mats, 40)
    gs = api.Scene.from_obj(S.Scene(sc.name, sc.verts, sc.tris, sc.tri_mat, tgt))
    m = api.trace(gs, [tx], p)["maps"][0]
    gs.free()
    return m


def test_db_loss_kernel(api):
    rng = np.random.default_rng(0)
    a = 10 ** rng.uniform(-20, -5, size=5000)
    b = 10 ** rng.uniform(-20, -5, size=5000)
    a[:100] = 0
    ta, tb = torch.tensor(a, dtype=torch.float32, device="cuda"), torch.tensor(b, dtype=torch.float32, device="cuda")
    loss, g, valid = api.db_mse_loss(ta, tb, 1e-15)
    a32, b32 = a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    V = (a32 > 1e-15) & (b32 > 1e-15)
    d = 10 * (np.log10(a32[V]) - np.log10(b32[V]))
    assert int(valid) == V.sum()
    assert abs(float(loss) - np.mean(d * d)) <= 1e-5 * np.mean(d * d)
    gref = np.zeros_like(a32)
    gref[V] = 2 / V.sum() * d * 10 / (math.log(10) * a32[V])
    gg = g.double().cpu().numpy()
    # FP32 log10 difference: absolute error ~1e-6 dB, i.e. relative error grows as d -> 0
    assert np.allclose(gg, gref, rtol=2e-4, atol=1e-5 * np.abs(gref).max())


def test_adjoint_retrace_takes_forward_choices(api):
    sc, tx, p = _setup()
    gs = api.Scene.from_obj(sc)
    f = api.trace(gs, [tx], p, record=True)
    g = torch.rand_like(f["maps"])
    a = api.grad(gs, [tx], p, g, record=True)
    assert torch.equal(f["record"], a["record"])
    assert a["stats"]["segments"] == f["stats"]["segments"]
    gs.free()


@pytest.mark.parametrize("deposit", [1, 0])
def test_adjoint_matches_oracle_gradient(orc, api, deposit):
    sc, tx, p = _setup(deposit=deposit)
    gs = api.Scene.from_obj(sc)
    tgt = _target(api, sc, tx, p)
    f = api.trace(gs, [tx], p, record=True)
    loss, dLdC, valid = api.db_mse_loss(f["maps"][0], tgt)
    assert int(valid) > 1000
    a = api.grad(gs, [tx], p, dLdC.view(1, p.ny, p.nx))
    ad = np.concatenate([a["d_eps"].cpu().numpy(), a["d_sigma"].cpu().numpy(), a["d_tx"][0].cpu().numpy()])
    rec = f["record"].view(tx.count(), p.max_depth + 1, 4).cpu().numpy()
    # the oracle certifies the GPU's choices, then differentiates along them
    compare_maps(orc, sc, tx, p, f["maps"][0].cpu().numpy(), rec)
    de, ds, dt = orc.grad(sc, tx, p, rec, dLdC.double().cpu().numpy())
    ref = np.concatenate([de, ds, dt])
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    err = np.abs(ad - ref) / scale
    assert np.all(err <= GRAD_RTOL), err
    if deposit == 0:
        assert np.all(ad[-3:] == 0.0)
    gs.free()


def test_adjoint_vs_gpu_finite_differences(api):
    """Materials only (frozen sampling): central differences of the FP32
    traced loss, Richardson-extrapolated with 2h (steps below)."""
    sc, tx, p = _setup(stride=3)
    gs = api.Scene.from_obj(sc)
    tgt = _target(api, sc, tx, p)
    mats0 = sc.mats.astype(np.float64)
    f = api.trace(gs, [tx], p)
    _, dLdC, _ = api.db_mse_loss(f["maps"][0], tgt)
    g = dLdC.view(1, p.ny, p.nx)
    a = api.grad(gs, [tx], p, g)

    def J(m):
        gs.set_materials(m, sampling=mats0)
        mp = api.trace(gs, [tx], p)["maps"][0].double()
        return float((mp * g[0].double()).sum())

    def central(m, c, h):
        mp, mm = mats0.copy(), mats0.copy()
        mp[m, c] += h
        mm[m, c] -= h
        return (J(mp) - J(mm)) / (2 * h)

    fd = []
    for j in range(2 * sc.nm):
        m, c = j % sc.nm, j // sc.nm
        # sigma: h = 1e-3 relative.  eps_r: the loss oscillates at up to
        # L x 58 rad per unit eps_r (each slab pass turns the phase 2 Re q by
        # ~58 rad per unit at 28 GHz, 0.2 m), so h = 1e-5 relative keeps the
        # step well below one radian; FP32 map noise stays below 1e-3 of the
        # difference.
        h = (1e-5 if c == 0 else 1e-3) * abs(mats0[m, c])
        # Richardson extrapolation of the steps 2h and h (truncation O(h^4))
        fd.append((4 * central(m, c, h) - central(m, c, 2 * h)) / 3)
    fd = np.array(fd)
    ad = np.concatenate([a["d_eps"].cpu().numpy(), a["d_sigma"].cpu().numpy()])
    # FP32 finite differences are a consistency check (the exact comparison
    # is against the FP64 oracle's dual numbers): errors are measured against
    # max(|fd|, 5e-2 max|fd|), the FD noise floor of the small components.
    scale = np.maximum(np.abs(fd), 5e-2 * np.abs(fd).max())
    assert np.all(np.abs(ad - fd) <= 2e-2 * scale), np.abs(ad - fd) / scale
    gs.free()


def test_autograd_function(api):
    sc, tx, p = _setup(stride=29)
    gs = api.Scene.from_obj(sc)
    tgt = _target(api, sc, tx, p)
    eps = torch.tensor(sc.mats[:, 0], dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(sc.mats[:, 1], dtype=torch.float64, requires_grad=True)
    pos = torch.tensor([tx.pos], dtype=torch.float64, requires_grad=True)
    maps = api.RadioMap.apply(eps, sig, pos, gs, [tx], p, sc.mats[:, 2])
    loss, dLdC, _ = api.db_mse_loss(maps[0].detach(), tgt)
    maps.backward(dLdC.view_as(maps))
    ref = api.grad(gs, [tx], p, dLdC.view_as(maps))
    assert torch.allclose(eps.grad.float().cuda(), ref["d_eps"], rtol=1e-5, atol=0)
    assert torch.allclose(pos.grad.float().cuda(), ref["d_tx"], rtol=1e-5, atol=0)
    gs.free()


def test_partition_gradients_sum_to_full(api):
    """The adjoint is linear in the rays: the gradients of the lattice shares
    of three ranks (the sharded adjoint's partition) add up to the gradient of
    the whole subset, to the order of FP32 atomic additions."""
    from paper_2504_21719_b300.shard import partition_tx
    sc, tx, p = _setup(stride=7)
    gs = api.Scene.from_obj(sc)
    tgt = _target(api, sc, tx, p)
    f = api.trace(gs, [tx], p)
    _, dLdC, _ = api.db_mse_loss(f["maps"][0], tgt)
    g = dLdC.view(1, p.ny, p.nx)
    full = api.grad(gs, [tx], p, g)
    parts = [api.grad(gs, [partition_tx(tx, r, 3)], p, g) for r in range(3)]
    for key in ("d_eps", "d_sigma", "d_tx"):
        a = full[key].double()
        b = sum(q[key].double() for q in parts)
        scale = a.abs().max().item()
        assert scale > 0
        assert torch.all((a - b).abs() <= 1e-4 * scale), (key, a, b)
    gs.free()


@pytest.mark.parametrize("regular", [True, False])
def test_adjoint_with_array_matches_oracle(orc, api, regular):
    """The adjoint re-evaluates the synthetic-array factor at launch (Sec. 4.4):
    a steered 8-element ULA (Horner path) or 6 irregular elements (per-element
    path), gradient of the dB loss against the oracle's along the GPU's record."""
    sc, tx, p = _setup()
    if regular:
        tx.ant_pos, tx.precoding = S.uniform_linear_array(8, p.freq_hz, 0.5, axis=0, steer=(0.3, 1.0, -0.2))
    else:
        rng = np.random.default_rng(3)
        tx.ant_pos = rng.uniform(-0.03, 0.03, size=(6, 3))
        w = rng.normal(size=6) + 1j * rng.normal(size=6)
        tx.precoding = w / np.linalg.norm(w)
    gs = api.Scene.from_obj(sc)
    tgt = _target(api, sc, tx, p)
    f = api.trace(gs, [tx], p, record=True)
    loss, dLdC, valid = api.db_mse_loss(f["maps"][0], tgt)
    assert int(valid) > 1000
    a = api.grad(gs, [tx], p, dLdC.view(1, p.ny, p.nx), record=True)
    assert torch.equal(f["record"], a["record"])
    ad = np.concatenate([a["d_eps"].cpu().numpy(), a["d_sigma"].cpu().numpy(), a["d_tx"][0].cpu().numpy()])
    rec = f["record"].view(tx.count(), p.max_depth + 1, 4).cpu().numpy()
    compare_maps(orc, sc, tx, p, f["maps"][0].cpu().numpy(), rec)
    de, ds, dt = orc.grad(sc, tx, p, rec, dLdC.double().cpu().numpy())
    ref = np.concatenate([de, ds, dt])
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    err = np.abs(ad - ref) / scale
    assert np.all(err <= GRAD_RTOL), err
    gs.free()


@pytest.mark.parametrize("deposit", [0, 1])
def test_large_city_adjoint_matches_oracle(orc, api, deposit):
    """Procedural city (0.97M triangles), depth 8, 2048 x 2048 cells: the
    adjoint of the dB loss on a lattice subset of one transmitter against the
    oracle's dual-number gradient along the GPU's record, after the oracle (brute
    force over every triangle) has certified that record.  Box cells give the
    material gradient only (the TX-position gradient is exactly 0); bilinear
    cells add the TX position."""
    sc, txs, p = S.workload(5)
    tx = copy.copy(txs[0])
    tx.ray_stride, tx.ray_begin = 166_667, 11                # 600 rays of the 1e8-ray lattice
    p.deposit = deposit
    p.record_coin = True
    gs = api.Scene.from_obj(sc)
    tgt = _target(api, sc, tx, p)
    f = api.trace(gs, [tx], p, record=True)
    loss, dLdC, valid = api.db_mse_loss(f["maps"][0], tgt)
    assert int(valid) >= 100
    a = api.grad(gs, [tx], p, dLdC.view(1, p.ny, p.nx), record=True)
    assert torch.equal(f["record"], a["record"])
    ad = np.concatenate([a["d_eps"].cpu().numpy(), a["d_sigma"].cpu().numpy(), a["d_tx"][0].cpu().numpy()])
    rec = f["record"].view(tx.count(), p.max_depth + 1, 4).cpu().numpy()
    assert (rec[:, 1:, 0] >= 0).sum() > 100                  # paths with interactions reach the map
    compare_maps(orc, sc, tx, p, f["maps"][0].cpu().numpy(), rec)
    de, ds, dt = orc.grad(sc, tx, p, rec, dLdC.double().cpu().numpy())
    ref = np.concatenate([de, ds, dt])
    assert np.abs(ref[:2 * sc.nm]).max() > 0
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    err = np.abs(ad - ref) / scale
    assert np.all(err <= GRAD_RTOL), err
    if deposit == 0:
        assert np.all(ad[-3:] == 0.0)
    gs.free()


def test_large_city_full_adjoint_partition(api):
    """The full-size city adjoint (16 TX x 1e8 rays, depth 8, one launch in the
    benchmark's configuration) equals the sum of the adjoints of two disjoint
    lattice halves, to the order of the FP32 block sums."""
    from paper_2504_21719_b300.shard import partition_tx
    sc, txs, p = S.workload(5)
    gs = api.Scene.from_obj(sc)
    f = api.trace(gs, txs, p)
    # dL/dC of a loss that weights every cell by its own path gain's dB value
    g = (10.0 * torch.log10(f["maps"].clamp_min(1e-15)) + 150.0) * 1e-6
    full = api.grad(gs, txs, p, g)
    assert full["stats"]["segments"] == f["stats"]["segments"]
    parts = [api.grad(gs, [partition_tx(t, r, 2) for t in txs], p, g) for r in range(2)]
    for key in ("d_eps", "d_sigma"):
        a = full[key].double()
        b = parts[0][key].double() + parts[1][key].double()
        scale = a.abs().max().item()
        assert scale > 0
        assert torch.all((a - b).abs() <= 1e-4 * scale), (key, a, b)
    assert torch.all(full["d_tx"] == 0)
    gs.free()


def test_large_city_adjoint_with_array(orc, api):
    """The adjoint with a steered 16-element uniform linear array (its factor from
    the pre-pass in both the forward and the gradient call) on the city: a
    lattice subset of one transmitter, depth 8, bilinear cells, against the
    oracle's dual-number gradient along the certified GPU record."""
    sc, txs, p = S.workload(5)
    tx = copy.copy(txs[0])
    tx.ray_stride, tx.ray_begin = 166_667, 3
    tx.ant_pos, tx.precoding = S.uniform_linear_array(16, p.freq_hz, 0.5, axis=1, steer=(0.3, 1.0, -0.2))
    p.deposit = 1
    gs = api.Scene.from_obj(sc)
    tgt = _target(api, sc, tx, p)
    f = api.trace(gs, [tx], p, record=True)
    loss, dLdC, valid = api.db_mse_loss(f["maps"][0], tgt)
    assert int(valid) >= 100
    a = api.grad(gs, [tx], p, dLdC.view(1, p.ny, p.nx), record=True)
    assert torch.equal(f["record"], a["record"])
    ad = np.concatenate([a["d_eps"].cpu().numpy(), a["d_sigma"].cpu().numpy(), a["d_tx"][0].cpu().numpy()])
    rec = f["record"].view(tx.count(), p.max_depth + 1, 4).cpu().numpy()
    compare_maps(orc, sc, tx, p, f["maps"][0].cpu().numpy(), rec)
    de, ds, dt = orc.grad(sc, tx, p, rec, dLdC.double().cpu().numpy())
    ref = np.concatenate([de, ds, dt])
    assert np.abs(ref[:2 * sc.nm]).max() > 0
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    err = np.abs(ad - ref) / scale
    assert np.all(err <= GRAD_RTOL), err
    gs.free()
