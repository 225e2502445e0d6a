"""GPU radio maps on a mesh measurement surface vs the FP64 oracle, after the
oracle replays the GPU's hits and decisions; crossings within tol of a
triangle's boundary are bounded by the oracle's per-cell slack."""
import copy

import numpy as np
import pytest
import torch

from synth import scenes as S
from gpu_helpers import compare_mesh, coin
from test_oracle_mesh import grid_surface

pytestmark = pytest.mark.gpu


def terrain(n=32, half=64.0):
    return grid_surface(-half, -half, 2 * half / n, n, n,
                        lambda X, Y: 1.5 + 0.5 * np.sin(X / 9.0) * np.cos(Y / 7.0))


def _run(api, sc, surf_v, surf_t, txs, p, builder="auto"):
    gs = api.Scene.from_obj(sc, builder=builder)
    su = api.surface(surf_v, surf_t, builder=builder)
    r = api.trace_mesh(gs, su, txs, coin(p), record=True)
    torch.cuda.synchronize()
    out = (r["maps"].cpu().numpy(), r["record"].cpu().numpy(), r["stats"])
    su.free()
    gs.free()
    return out


@pytest.mark.parametrize("stride,begin,builder", [(997, 0, "auto"), (1009, 5, "sah")])
def test_mesh_parity_manhattan(orc, api, stride, begin, builder):
    """builder "sah": the scene and the surface both walk binned-SAH trees."""
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride, tx.ray_begin = stride, begin
    V, T = terrain()
    m, rec, st = _run(api, sc, V, T, [tx], p, builder)
    assert st["rays"] == tx.count() and st["deposits"] > 1000
    info = compare_mesh(orc, sc, tx, p, V, T, m[0], rec)
    assert info["cells"] > 1000


def test_mesh_parity_diffuse_dual_pol(orc, api):
    sc, txs, p = S.workload(2)
    sc = sc.with_scattering(0.5, 0.2, np.arange(sc.nm) % 3, 3, 2, 0.6)
    p = copy.copy(p)
    p.diffuse = True
    tx = txs[0]
    tx.ray_stride, tx.pol = 1499, 2
    V, T = terrain(24, 80.0)
    m, rec, st = _run(api, sc, V, T, [tx], p)
    info = compare_mesh(orc, sc, tx, p, V, T, m[0], rec)
    assert info["cells"] > 500


def test_mesh_batched_equals_single(api):
    sc, _, p = S.workload(2)
    txs = [S.Tx(pos=pos, num_rays=n, seed=i) for i, (pos, n) in
           enumerate((((0.0, 0.0, 30.0), 200_000), ((40.0, -30.0, 25.0), 150_000), ((-60.0, 20.0, 35.0), 250_000)))]
    V, T = terrain(40, 120.0)
    gs = api.Scene.from_obj(sc)
    su = api.surface(V, T)
    both = api.trace_mesh(gs, su, txs, p)["maps"].double()
    for i, t in enumerate(txs):
        one = api.trace_mesh(gs, su, [t], p)["maps"][0].double()
        mask = one > 1e-15
        assert mask.sum() > 100
        assert torch.all((both[i] - one).abs()[mask] <= 2e-5 * one[mask])
    su.free()
    gs.free()


def test_mesh_rejects_bilinear(api):
    sc, txs, p = S.workload(1)
    V, T = terrain(4, 10.0)
    gs = api.Scene.from_obj(sc)
    su = api.surface(V, T)
    q = copy.copy(p)
    q.deposit = 1
    with pytest.raises(RuntimeError, match="box cells"):
        api.trace_mesh(gs, su, txs, q)
    su.free()
    gs.free()


@pytest.mark.parametrize("diffuse", [False, True])
def test_mesh_adjoint_matches_oracle_gradient(orc, api, diffuse):
    """The mesh adjoint against the oracle's dual-number gradient along the
    GPU's own record (after the oracle certified the forward's choices); the
    TX-position gradient of box cells is zero."""
    sc, txs, p = S.workload(4)
    tx = txs[0]
    tx.ray_stride = 13
    p.deposit = 0
    if diffuse:
        sc = sc.with_scattering(np.linspace(0.2, 0.8, sc.nm), 0.3, np.arange(sc.nm) % 3, 2, 3, 0.5)
        p = copy.copy(p)
        p.diffuse = True
    V, T = terrain(48, 60.0)
    gs = api.Scene.from_obj(sc)
    su = api.surface(V, T)
    f = api.trace_mesh(gs, su, [tx], p, record=True)
    rec = f["record"].view(tx.count(), p.max_depth + 1, 4).cpu().numpy()
    compare_mesh(orc, sc, tx, p, V, T, f["maps"][0].cpu().numpy(), rec)
    g = torch.from_numpy(np.random.default_rng(9).uniform(0.0, 1.0, (1, len(T))).astype(np.float32)).cuda()
    a = api.grad_mesh(gs, su, [tx], p, g, record=True)
    assert torch.equal(a["record"], f["record"])
    ad = np.concatenate([a["d_eps"].cpu().numpy(), a["d_sigma"].cpu().numpy()])
    de, ds, dt = orc.grad_mesh(sc, tx, p, V, T, rec, g[0].double().cpu().numpy())
    ref = np.concatenate([de, ds])
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    err = np.abs(ad - ref) / scale
    assert np.all(err <= 1e-2), err
    assert torch.all(a["d_tx"] == 0.0) and np.all(dt == 0.0)
    su.free()
    gs.free()


def test_mesh_edge_cases(orc, api):
    """Free space over a one-triangle surface (a large-triangle list of one,
    no tree), a two-triangle surface, and an empty ray subset."""
    sc = S.empty_scene()
    tx = S.Tx(pos=(0.3, -0.2, 10.0), num_rays=200_000, seed=1)
    p = S.TraceParams(3.5e9, 0)
    for V, T in ((np.array([[-30, -30, 1.5], [30, -30, 1.0], [0, 40, 2.0]], np.float32), np.array([[0, 1, 2]], np.int32)),
                 terrain(1, 25.0)):
        m, rec, st = _run(api, sc, V, T, [tx], p)
        assert st["deposits"] > 1000
        compare_mesh(orc, sc, tx, p, V, T, m[0], rec)
    gs = api.Scene.from_obj(sc)
    su = api.surface(*terrain(2, 10.0))
    r = api.trace_mesh(gs, su, [S.Tx(pos=(0, 0, 5.0), num_rays=1000, ray_count=0)], p)
    assert r["stats"]["rays"] == 0 and float(r["maps"].abs().sum()) == 0.0
    su.free()
    gs.free()


def test_mesh_parity_city(orc, api):
    """The largest scene: a rolling 256 m x 256 m measurement surface (8192
    triangles) around one transmitter of the 0.97M-triangle city (depth 8), a
    sampled lattice subset of its rays, replayed by the oracle."""
    sc, txs, p = S.workload(5)
    tx = copy.copy(txs[0])
    tx.ray_stride, tx.ray_begin = 99_991, 3
    V, T = grid_surface(tx.pos[0] - 128.0, tx.pos[1] - 128.0, 4.0, 64, 64,
                        lambda X, Y: 1.5 + 0.5 * np.sin(X / 9.0) * np.cos(Y / 7.0))
    m, rec, st = _run(api, sc, V, T, [tx], p)
    assert st["rays"] == tx.count() and st["deposits"] > 300
    info = compare_mesh(orc, sc, tx, p, V, T, m[0], rec)
    assert info["cells"] > 300


def test_mesh_adjoint_city(orc, api):
    """The mesh adjoint on the largest scene: a 4096-triangle rolling surface
    around one transmitter of the 0.97M-triangle city (depth 8), a sampled
    lattice subset of its rays, against the oracle's dual-number gradient along
    the GPU's certified record; the re-trace takes the forward's choices."""
    sc, txs, p = S.workload(5)
    tx = copy.copy(txs[0])
    tx.ray_stride, tx.ray_begin = 199_999, 5
    V, T = grid_surface(tx.pos[0] - 96.0, tx.pos[1] - 96.0, 6.0, 32, 64,
                        lambda X, Y: 1.5 + 0.5 * np.sin(X / 9.0) * np.cos(Y / 7.0))
    gs = api.Scene.from_obj(sc)
    su = api.surface(V, T)
    f = api.trace_mesh(gs, su, [tx], p, record=True)
    rec = f["record"].view(tx.count(), p.max_depth + 1, 4).cpu().numpy()
    info = compare_mesh(orc, sc, tx, p, V, T, f["maps"][0].cpu().numpy(), rec)
    assert info["cells"] > 100
    g = torch.from_numpy(np.random.default_rng(9).uniform(0.0, 1.0, (1, len(T))).astype(np.float32)).cuda()
    a = api.grad_mesh(gs, su, [tx], p, g, record=True)
    assert torch.equal(a["record"], f["record"])
    ad = np.concatenate([a["d_eps"].cpu().numpy(), a["d_sigma"].cpu().numpy()])
    de, ds, dt = orc.grad_mesh(sc, tx, p, V, T, rec, g[0].double().cpu().numpy())
    ref = np.concatenate([de, ds])
    assert np.abs(ref).max() > 0
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    err = np.abs(ad - ref) / scale
    assert np.all(err <= 1e-2), err
    su.free()
    gs.free()
