"""GPU parity of the first-order diffraction radio map (Sec. 4, "Computation
of Radio Map due to Diffraction"; UTD of App. A.8): the library's wedges
against the oracle's, and the maps, replay-checked against the FP64 oracle."""
import numpy as np
import pytest
import torch

from synth import scenes as S
from gpu_helpers import compare_diffraction

pytestmark = pytest.mark.gpu


def _wedge_array(w, n):
    return np.array([[*x.origin, *x.edge, *x.n0, *x.nn, x.length, x.n, x.tri0, x.trin] for x in w[:n]])


@pytest.mark.parametrize("scene", ["box", "manhattan"])
def test_wedges_match_oracle(orc, api, scene):
    sc = S.single_box(ground=500.0) if scene == "box" else S.workload(2)[0]
    gs = api.Scene.from_obj(sc)
    w, n = gs.wedges()
    got = _wedge_array(w, n)
    ref = orc.wedges(sc)
    assert got.shape == ref.shape
    assert np.array_equal(got[:, 14:16], ref[:, 14:16])
    assert np.allclose(got[:, :14], ref[:, :14], rtol=1e-6, atol=1e-5)
    gs.free()


def _run(api, sc, tx, p, ns, builder="auto"):
    gs = api.Scene.from_obj(sc, builder=builder)
    r = api.diffraction_map(gs, [tx], p, ns, record=True)
    torch.cuda.synchronize()
    out = (r["maps"][0].cpu().numpy(), r["record"].cpu().numpy(), r["stats"])
    gs.free()
    return out


def test_diffraction_parity_single_box(orc, api):
    sc = S.single_box(ground=500.0)
    p = S.TraceParams(3.5e9, 0, cell_size=2.0, nx=60, ny=60, map_origin=(10.0, 15.0, 1.5))
    tx = S.Tx(pos=(-30.0, -20.0, 15.0), num_rays=1)
    m, rec, st = _run(api, sc, tx, p, 4096)
    assert st["deposits"] > 5000 and st["rays"] == len(rec)
    compare_diffraction(orc, sc, tx, p, 4096, m, rec)


@pytest.mark.parametrize("pol,pattern,deposit,builder", [(0, 0, 0, "auto"), (2, 1, 1, "auto"), (0, 0, 1, "sah")])
def test_diffraction_parity_manhattan(orc, api, pol, pattern, deposit, builder):
    """builder "sah": the visibility queries walk the binned-SAH tree of the scene."""
    sc, txs, p = S.workload(2)
    p.nx = p.ny = 256
    p.cell_size = 2.0
    p.deposit = deposit
    tx = txs[0]
    tx.pol, tx.pattern = pol, pattern
    m, rec, st = _run(api, sc, tx, p, 256, builder)
    assert st["deposits"] > 5000
    compare_diffraction(orc, sc, tx, p, 256, m, rec)


def test_diffraction_batched_transmitters_match_single(api):
    sc, txs, p = S.workload(2)
    p.nx = p.ny = 128
    p.cell_size = 4.0
    a = S.Tx(pos=(0.0, 0.0, 30.0), num_rays=1)
    b = S.Tx(pos=(-75.0, 32.0, 12.0), num_rays=1, pol=1)
    gs = api.Scene.from_obj(sc)
    both = api.diffraction_map(gs, [a, b], p, 128)["maps"].cpu().numpy()
    for k, t in enumerate((a, b)):
        one = api.diffraction_map(gs, [t], p, 128)["maps"][0].cpu().numpy()
        assert np.allclose(both[k], one, rtol=1e-6, atol=1e-6 * one.max())
    gs.free()


def test_diffraction_rejects_bad_arguments(api):
    from paper_2504_21719_b300 import _lib as L
    sc = S.single_box()
    gs = api.Scene.from_obj(sc)
    w, n = gs.wedges()
    p = api.params_from(S.TraceParams(3.5e9, 0))
    arr, ntx = api._tx_array([S.Tx(pos=(-30.0, -20.0, 15.0), num_rays=1)])
    maps = torch.empty((1, 100, 100), dtype=torch.float32, device="cuda")
    lib = L.load()
    st = L.rm_stats()
    import ctypes as C
    assert lib.rm_diffraction_map(gs.handle, w, n, arr, ntx, C.byref(p), 0, maps.data_ptr(), C.byref(st), None,
                                  None) == L.RM_EINVAL
    bad = (L.rm_wedge * 1)()
    bad[0] = w[0]
    bad[0].n = 2.5
    assert lib.rm_diffraction_map(gs.handle, bad, 1, arr, ntx, C.byref(p), 16, maps.data_ptr(), C.byref(st), None,
                                  None) == L.RM_EINVAL
    assert b"wedge 0" in lib.rm_last_error()
    gs.free()


@pytest.mark.parametrize("which", ["box", "manhattan"])
def test_diffraction_mesh_parity(orc, api, which):
    """The diffraction map on a rolling mesh surface vs the oracle's replay."""
    import numpy as np
    from gpu_helpers import compare_diffraction_mesh
    from test_oracle_mesh import grid_surface
    if which == "box":
        sc = S.single_box(ground=500.0)
        tx = S.Tx(pos=(-30.0, -20.0, 15.0), num_rays=1)
        V, T = grid_surface(-50.0, -40.0, 4.0, 30, 30, lambda X, Y: 1.5 + 0.4 * np.sin(X / 6.0) * np.cos(Y / 5.0))
        spw = 2048
    else:
        sc, txs, _ = S.workload(2)
        tx = txs[0]
        V, T = grid_surface(-100.0, -100.0, 5.0, 40, 40, lambda X, Y: 1.5 + 0.5 * np.sin(X / 9.0) * np.cos(Y / 7.0))
        spw = 256
    p = S.TraceParams(3.5e9, 0)
    gs = api.Scene.from_obj(sc)
    su = api.surface(V, T)
    r = api.diffraction_map_mesh(gs, su, [tx], p, spw, record=True)
    torch.cuda.synchronize()
    st = r["stats"]
    assert st["deposits"] > 1000
    info = compare_diffraction_mesh(orc, sc, tx, p, spw, V, T, r["maps"][0].cpu().numpy(), r["record"].cpu().numpy())
    assert info["cells"] > 300
    q = S.TraceParams(3.5e9, 0, deposit=1)
    with pytest.raises(RuntimeError, match="box cells"):
        api.diffraction_map_mesh(gs, su, [tx], q, 16)
    su.free()
    gs.free()


@pytest.mark.parametrize("regular", [True, False])
def test_diffraction_parity_with_array(orc, api, regular):
    """The diffraction map's antenna field includes the synthetic-array factor
    at the direction to each wedge sample (Sec. 4.4): a steered 4-element ULA or
    5 irregular elements with complex precoding, single box at 3.5 GHz."""
    sc = S.single_box(ground=500.0)
    p = S.TraceParams(3.5e9, 0, cell_size=2.0, nx=60, ny=60, map_origin=(10.0, 15.0, 1.5))
    tx = S.Tx(pos=(-30.0, -20.0, 15.0), num_rays=1)
    if regular:
        tx.ant_pos, tx.precoding = S.uniform_linear_array(4, p.freq_hz, 0.5, axis=2, steer=(1.0, 0.8, -0.3))
    else:
        rng = np.random.default_rng(8)
        tx.ant_pos = rng.uniform(-0.1, 0.1, size=(5, 3))
        w = rng.normal(size=5) + 1j * rng.normal(size=5)
        tx.precoding = w / np.linalg.norm(w)
    m, rec, st = _run(api, sc, tx, p, 4096)
    assert st["deposits"] > 5000
    compare_diffraction(orc, sc, tx, p, 4096, m, rec)


def test_diffraction_parity_city_wedge_subset(orc, api):
    """The largest scene: the 0.97M-triangle city's wedges equal the oracle's,
    and a subset of them (300 within 80 m of the transmitter, 100 anywhere, in
    shuffled order) gives the oracle's visibility bits, cells and map.  The
    visibility queries walk the binned-SAH tree of the whole city."""
    from paper_2504_21719_b300 import _lib as L
    sc, txs, p = S.workload(5)
    tx = txs[0]
    gs = api.Scene.from_obj(sc)
    w, nw = gs.wedges()
    raw = np.frombuffer(w, dtype=np.float32).reshape(-1, 18)[:nw]      # 14 floats, then tri0 trin mat0 matn
    got = np.concatenate([raw[:, :14].astype(np.float64), raw[:, 14:16].view(np.int32).astype(np.float64)], 1)
    ref = orc.wedges(sc)
    assert got.shape == ref.shape and nw > 500_000
    assert np.array_equal(got[:, 14:16], ref[:, 14:16])
    assert np.allclose(got[:, :14], ref[:, :14], rtol=1e-6, atol=1e-4)
    rng = np.random.default_rng(21)
    near = np.flatnonzero(np.linalg.norm(ref[:, :2] - np.asarray(tx.pos[:2]), axis=1) < 80.0)
    idx = np.concatenate([rng.choice(near, 300, replace=False), rng.choice(nw, 100, replace=False)])
    rng.shuffle(idx)
    sub = (L.rm_wedge * len(idx))(*[w[int(i)] for i in idx])
    ns = 16
    r = api.diffraction_map(gs, [tx], p, ns, wedges=(sub, len(idx)), record=True)
    torch.cuda.synchronize()
    rec = r["record"].cpu().numpy()
    assert (rec[:, 0] == 0).sum() > 200 and (rec[:, 0] > 0).sum() > 1000   # visible and blocked samples
    compare_diffraction(orc, sc, tx, p, ns, r["maps"][0].cpu().numpy(), rec, wedge_index=idx)
    gs.free()


@pytest.mark.parametrize("nsel,ns,ntx", [(0, 16, 1), (1, 1, 1), (1, 3, 1), (7, 5, 1), (13, 37, 2), (41, 129, 3)])
def test_diffraction_ragged_sizes(orc, api, nsel, ns, ntx):
    """Totals that fill no warp, or leave ragged tails of the kernel's 32-sample
    batches and 128-sample queue chunks (ntx * nsel * ns = 0, 1, 3, 35, 962,
    15867), and several transmitters in one launch: the records and maps of
    every transmitter replay against the oracle; no wedges give empty maps."""
    from paper_2504_21719_b300 import _lib as L
    sc, txs, p = S.workload(2)
    p.nx = p.ny = 256
    p.cell_size = 2.0
    gs = api.Scene.from_obj(sc)
    w, nw = gs.wedges()
    ref = _wedge_array(w, nw)
    # wedges near the first transmitter, so that some samples are lit and visible
    near = np.argsort(np.linalg.norm(ref[:, :2] - np.asarray(txs[0].pos[:2]), axis=1))
    idx = np.random.default_rng(nsel).permutation(near[:200])[:nsel]
    sub = (L.rm_wedge * max(nsel, 1))(*[w[int(i)] for i in idx])
    tl = [txs[0], S.Tx(pos=(-75.0, 32.0, 12.0), num_rays=1, pol=1), S.Tx(pos=(40.0, -90.0, 25.0), num_rays=1)][:ntx]
    r = api.diffraction_map(gs, tl, p, ns, wedges=(sub, nsel), record=True)
    torch.cuda.synchronize()
    assert r["stats"]["rays"] == ntx * nsel * ns
    maps = r["maps"].cpu().numpy()
    if nsel == 0:
        assert not maps.any()
    else:
        rec = r["record"].cpu().numpy().reshape(ntx, nsel * ns, 4)
        for k, t in enumerate(tl):
            compare_diffraction(orc, sc, t, p, ns, maps[k], rec[k], wedge_index=idx)
    gs.free()


def test_diffraction_mesh_city_wedge_subset(orc, api):
    """The mesh-surface diffraction map on the largest scene: 300 wedges within
    80 m of a city transmitter (16 samples each) onto a 4096-triangle surface
    around it, replayed against the oracle through the city's SAH tree."""
    from paper_2504_21719_b300 import _lib as L
    from gpu_helpers import compare_diffraction_mesh
    from test_oracle_mesh import grid_surface
    sc, txs, p = S.workload(5)
    tx = txs[0]
    gs = api.Scene.from_obj(sc)
    w, nw = gs.wedges()
    raw = np.frombuffer(w, dtype=np.float32).reshape(-1, 18)[:nw]
    near = np.flatnonzero(np.linalg.norm(raw[:, :2].astype(np.float64) - np.asarray(tx.pos[:2]), axis=1) < 80.0)
    idx = np.random.default_rng(22).permutation(near)[:300]
    sub = (L.rm_wedge * len(idx))(*[w[int(i)] for i in idx])
    V, T = grid_surface(tx.pos[0] - 96.0, tx.pos[1] - 96.0, 6.0, 32, 64,
                        lambda X, Y: 1.5 + 0.5 * np.sin(X / 9.0) * np.cos(Y / 7.0))
    su = api.surface(V, T)
    ns = 16
    r = api.diffraction_map_mesh(gs, su, [tx], p, ns, wedges=(sub, len(idx)), record=True)
    torch.cuda.synchronize()
    rec = r["record"].cpu().numpy()
    assert (rec[:, 0] == 0).sum() > 200 and r["stats"]["deposits"] > 50
    compare_diffraction_mesh(orc, sc, tx, p, ns, V, T, r["maps"][0].cpu().numpy(), rec, wedge_index=idx)
    su.free()
    gs.free()
