"""The adjoint that replays the forward's recorded closest hits
(rm_radio_map_trace_hits, rm_radio_map_grad_hits) against the re-tracing
adjoint: the same segment records, the same gradients up to the order of their
atomic sums, no node visited; the recorded hits against the debug record; the
length check and the fallback to the traversal."""
import copy

import numpy as np
import pytest
import torch

from synth import scenes as S

pytestmark = pytest.mark.gpu


def _compare_grads(a, b):
    for key in ("d_eps", "d_sigma", "d_tx"):
        x, y = a[key].double(), b[key].double()
        scale = max(x.abs().max().item(), 1e-30)
        assert torch.all((x - y).abs() <= 1e-5 * scale), (key, x, y)


def _replay_equals_retrace(api, sc, tx, p, builder="auto"):
    gs = api.Scene.from_obj(sc, builder=builder)
    f = api.trace(gs, [tx], p, keep_hits=True)
    # the recording forward (its own instantiation of the plain tracer) gives the plain
    # tracer's maps, up to the order of the FP64 sums
    plain = api.trace(gs, [tx], p)
    assert f["stats"]["segments"] == plain["stats"]["segments"]
    assert f["stats"]["deposits"] == plain["stats"]["deposits"]
    assert torch.allclose(f["maps"], plain["maps"], rtol=1e-6, atol=0)
    # and takes the record's paths (the instantiations' approximate divisions may round a
    # few ulps apart, so the deposits agree to 1e-5)
    fr = api.trace(gs, [tx], p, record=True)
    assert f["stats"]["segments"] == fr["stats"]["segments"]
    assert f["stats"]["deposits"] == fr["stats"]["deposits"]
    assert torch.allclose(f["maps"], fr["maps"], rtol=1e-5, atol=0)
    g = (10.0 * torch.log10(f["maps"].clamp_min(1e-15)) + 150.0) * 1e-6
    ref = api.grad(gs, [tx], p, g, record=True)
    rep = api.grad(gs, [tx], p, g, record=True, hits=f["hits"])
    assert torch.equal(ref["record"], rep["record"])
    assert rep["stats"]["segments"] == ref["stats"]["segments"]
    assert ref["stats"]["nodes_visited"] > 0 and rep["stats"]["nodes_visited"] == 0
    _compare_grads(ref, rep)
    assert ref["d_eps"].abs().max() > 0
    gs.free()


@pytest.mark.parametrize("deposit", [0, 1])
def test_replay_equals_retrace_differentiable(api, deposit):
    sc, txs, p = S.workload(4)
    tx = txs[0]
    tx.ray_stride = 7
    p.deposit = deposit
    _replay_equals_retrace(api, sc, tx, p)


def test_replay_equals_retrace_diffuse(api):
    sc, txs, p = S.workload(4)
    sc = sc.with_scattering(0.4, 0.2, np.arange(sc.nm) % 3, 3, 2, 0.6)
    tx = txs[0]
    tx.ray_stride = 11
    p.diffuse = True
    _replay_equals_retrace(api, sc, tx, p)


def test_replay_equals_retrace_city(api):
    """The 0.97M-triangle city on its binned-SAH tree, depth 8, a 1e4-ray subset."""
    sc, txs, p = S.workload(5)
    tx = copy.copy(txs[2])
    tx.ray_stride, tx.ray_begin = 9973, 5
    _replay_equals_retrace(api, sc, tx, p)


def test_replay_equals_retrace_city_full(api):
    """The benchmark's full city workload (16 TX x 1e8 rays, depth 8, one launch):
    the adjoint replaying the 6.3e9 recorded hits (57.6 GB) gives the re-tracing
    adjoint's segments and gradients, to the order of the FP32 block sums."""
    sc, txs, p = S.workload(5)
    gs = api.Scene.from_obj(sc)
    f = api.trace(gs, txs, p, keep_hits=True)
    g = (10.0 * torch.log10(f["maps"].clamp_min(1e-15)) + 150.0) * 1e-6
    rep = api.grad(gs, txs, p, g, hits=f.pop("hits"))
    ref = api.grad(gs, txs, p, g)
    assert rep["stats"]["segments"] == ref["stats"]["segments"] == f["stats"]["segments"]
    assert rep["stats"]["deposits"] == ref["stats"]["deposits"]
    for key in ("d_eps", "d_sigma"):
        a, b = ref[key].double(), rep[key].double()
        scale = a.abs().max().item()
        assert scale > 0
        assert torch.all((a - b).abs() <= 1e-4 * scale), (key, a, b)
    gs.free()


def test_hits_are_the_records_hits(api):
    """hits[l, w] (depth l, work item w in the tracer's visit order) holds the leaf
    slots of the record's triangles at depth l (order[slot] = prim), -1 where the
    record says escaped, per depth the same multiset; depths a ray never reached
    keep what the buffer held."""
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 97
    gs = api.Scene.from_obj(sc)
    f = api.trace(gs, [tx], p, keep_hits=True)
    h = f["hits"].fill_(-7)
    f = api.trace(gs, [tx], p, keep_hits=True, hits_out=h)
    h = f["hits"].cpu().numpy().reshape(p.max_depth + 1, -1)
    rec = api.trace(gs, [tx], p, record=True)["record"].cpu().numpy()
    order = gs.export_bvh()["order"]
    prim = rec[:, 0].reshape(-1, p.max_depth + 1)
    assert (prim != -2).sum() > 10000
    for l in range(p.max_depth + 1):
        reached = prim[:, l] != -2
        got = h[l][h[l] != -7]
        assert len(got) == reached.sum()
        want = np.where(prim[reached, l] >= 0, 0, -1)
        hit = got >= 0
        assert np.array_equal(np.sort(np.where(hit, 0, -1)), np.sort(want))
        assert np.array_equal(np.sort(order[got[hit]]), np.sort(prim[reached, l][prim[reached, l] >= 0]))
    gs.free()


def test_short_or_foreign_hits(api):
    """A buffer shorter than rays x (L + 1) is RM_EINVAL; slots outside the scene
    fall back to the traversal, which gives the re-traced adjoint."""
    from paper_2504_21719_b300 import _lib as L
    sc, txs, p = S.workload(4)
    tx = txs[0]
    tx.ray_stride = 13
    gs = api.Scene.from_obj(sc)
    f = api.trace(gs, [tx], p, keep_hits=True)
    g = torch.full_like(f["maps"], 1e-6)
    with pytest.raises(api.RmError) as e:
        api.grad(gs, [tx], p, g, hits=f["hits"][:-1])
    assert e.value.status == L.RM_EINVAL
    foreign = torch.full_like(f["hits"], 1 << 30)
    ref = api.grad(gs, [tx], p, g, record=True)
    rep = api.grad(gs, [tx], p, g, record=True, hits=foreign)
    assert torch.equal(ref["record"], rep["record"])
    assert rep["stats"]["nodes_visited"] == ref["stats"]["nodes_visited"] > 0
    _compare_grads(ref, rep)
    gs.free()


def test_autograd_function_keeps_hits(api):
    """RadioMap with keep_hits: the same maps, and the backward's replayed
    gradients equal those of the re-tracing backward."""
    sc, txs, p = S.workload(4)
    tx = txs[0]
    tx.ray_stride = 17
    gs = api.Scene.from_obj(sc)
    res = []
    for keep in (False, True):
        eps = torch.tensor(sc.mats[:, 0], dtype=torch.float64, requires_grad=True)
        sig = torch.tensor(sc.mats[:, 1], dtype=torch.float64, requires_grad=True)
        pos = torch.tensor([tx.pos], dtype=torch.float64, requires_grad=True)
        maps = api.RadioMap.apply(eps, sig, pos, gs, [tx], p, sc.mats[:, 2], keep)
        g = (10.0 * torch.log10(maps.detach().clamp_min(1e-15)) + 150.0) * 1e-6
        maps.backward(g)
        res.append({"maps": maps.detach(), "d_eps": eps.grad, "d_sigma": sig.grad, "d_tx": pos.grad})
    assert torch.allclose(res[0]["maps"], res[1]["maps"], rtol=1e-5, atol=0)
    _compare_grads(res[0], res[1])
    assert res[0]["d_eps"].abs().max() > 0
    gs.free()


def test_hits_empty_and_depth_zero(api):
    """Edge cases: a transmitter with no rays (nothing recorded, zero gradients)
    beside one with rays, and max_depth 0 (one recorded slot per ray)."""
    sc, txs, p = S.workload(4)
    gs = api.Scene.from_obj(sc)
    empty = copy.copy(txs[0])
    empty.ray_count = 0
    f = api.trace(gs, [empty], p, keep_hits=True)
    assert f["stats"]["segments"] == 0 and torch.all(f["maps"] == 0)
    r = api.grad(gs, [empty], p, torch.ones_like(f["maps"]), hits=f["hits"])
    assert torch.all(r["d_eps"] == 0) and r["stats"]["segments"] == 0
    tx = copy.copy(txs[0])
    tx.ray_stride = 19
    both = [empty, tx]
    f2 = api.trace(gs, both, p, keep_hits=True)
    g2 = (10.0 * torch.log10(f2["maps"].clamp_min(1e-15)) + 150.0) * 1e-6
    _compare_grads(api.grad(gs, both, p, g2), api.grad(gs, both, p, g2, hits=f2["hits"]))
    p0 = copy.copy(p)
    p0.max_depth = 0
    f0 = api.trace(gs, [tx], p0, keep_hits=True)
    assert f0["hits"].numel() == api.tx_count(api.tx_from(tx))
    g0 = (10.0 * torch.log10(f0["maps"].clamp_min(1e-15)) + 150.0) * 1e-6
    ref = api.grad(gs, [tx], p0, g0, record=True)
    rep = api.grad(gs, [tx], p0, g0, record=True, hits=f0["hits"])
    assert torch.equal(ref["record"], rep["record"])
    _compare_grads(ref, rep)
    gs.free()


@pytest.mark.parametrize("diffuse", [False, True])
def test_mesh_replay_equals_retrace(api, diffuse):
    """Maps on a mesh measurement surface: the recording forward gives the plain
    mesh maps, and the mesh adjoint replaying its scene hits gives the re-tracing
    adjoint's records and gradients with no scene node visited."""
    sc, txs, p = S.workload(4)
    tx = copy.copy(txs[0])
    tx.ray_stride = 13
    p = copy.copy(p)
    p.deposit = 0
    if diffuse:
        sc = sc.with_scattering(np.linspace(0.2, 0.8, sc.nm), 0.3, np.arange(sc.nm) % 3, 2, 3, 0.5)
        p.diffuse = True
    n = 48
    x = np.linspace(-60.0, 60.0, n + 1)
    X, Y = np.meshgrid(x, x, indexing="xy")
    V = np.stack([X.ravel(), Y.ravel(), 1.5 + 0.5 * np.sin(X.ravel() / 9.0) * np.cos(Y.ravel() / 7.0)], 1)
    q = (np.arange(n)[None, :] + (n + 1) * np.arange(n)[:, None]).ravel()
    T = np.concatenate([np.stack([q, q + 1, q + n + 2], 1), np.stack([q, q + n + 2, q + n + 1], 1)])
    gs = api.Scene.from_obj(sc)
    su = api.surface(V.astype(np.float32), T.astype(np.int32))
    f = api.trace_mesh(gs, su, [tx], p, keep_hits=True)
    plain = api.trace_mesh(gs, su, [tx], p)
    assert f["stats"]["segments"] == plain["stats"]["segments"]
    assert torch.allclose(f["maps"], plain["maps"], rtol=1e-5, atol=0)
    g = torch.from_numpy(np.random.default_rng(9).uniform(0.0, 1.0, (1, len(T))).astype(np.float32)).cuda()
    ref = api.grad_mesh(gs, su, [tx], p, g, record=True)
    rep = api.grad_mesh(gs, su, [tx], p, g, record=True, hits=f["hits"])
    assert torch.equal(ref["record"], rep["record"])
    assert ref["stats"]["nodes_visited"] > 0 and rep["stats"]["nodes_visited"] == 0
    _compare_grads(ref, rep)
    assert ref["d_eps"].abs().max() > 0
    su.free()
    gs.free()
