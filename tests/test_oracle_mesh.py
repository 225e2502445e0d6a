"""Pins of the oracle's mesh-based measurement surface (Sec. 4, practical
notes): every triangle of a separate mesh is a cell, and a crossing adds
4 pi / (N A_i) (lambda0 / 4 pi)^2 |E|^2 / (|n_i . k| Pr) to it -- the planar
estimator (Eq. radio-map-solver-ci-all-2-estimator) with the cell's own area
and normal in the change of variables dA = r^2 / |n . k| d omega."""
import math

import numpy as np
import pytest

from synth import scenes as S
from closed_forms import C0


def grid_surface(x0, y0, cell, nx, ny, height):
    """Triangles of an nx x ny grid (two per cell, lower-right first) with
    vertex heights height(X, Y); the surface cells of planar cell (iy, ix) are
    2 * (iy * nx + ix) and the one after it."""
    xs = x0 + cell * np.arange(nx + 1)
    ys = y0 + cell * np.arange(ny + 1)
    X, Y = np.meshgrid(xs, ys)
    V = np.stack([X.ravel(), Y.ravel(), height(X, Y).ravel()], 1).astype(np.float32)
    T = []
    for iy in range(ny):
        for ix in range(nx):
            a = iy * (nx + 1) + ix
            T += [[a, a + 1, a + nx + 2], [a, a + nx + 2, a + nx + 1]]
    return V, np.array(T, np.int32)


def flat(z):
    return lambda X, Y: np.full(X.shape, z)


@pytest.mark.parametrize("which", ["two-ray", "manhattan"])
def test_flat_mesh_equals_planar_map(orc, which):
    """A flat mesh whose triangle pairs tile the planar map's cells gives the
    planar map: each crossing falls into exactly one triangle of its cell, and
    the triangle's area is half the cell's, so the mean of a pair equals the
    cell (to 5e-6: the surface's vertices are FP32, so at |x| ~ 130 m a 4 m
    cell's triangles differ in area from half the cell by a few 1e-6)."""
    if which == "two-ray":
        sc, txs, p = S.workload(1)
        tx = txs[0]
        tx.pos = (0.3, -0.2, 10.0)     # no lattice ray through a mesh vertex
        tx.num_rays = 200_000
        p.nx = p.ny = 20
        p.cell_size = 2.0
    else:
        sc, txs, p = S.workload(2)
        tx = txs[0]
        tx.ray_stride, tx.ray_count = 997, 10_000
        p.nx = p.ny = 64
        p.cell_size = 4.0
        p.map_origin = (1.3, -0.7, 1.5)
    x0, y0 = p.map_corner()
    V, T = grid_surface(x0, y0, p.cell_size, p.nx, p.ny, flat(p.map_origin[2]))
    m = orc.radio_map_mesh(sc, tx, p, V, T)["map"].reshape(p.ny, p.nx, 2)
    pl = orc.radio_map(sc, tx, p)["map"]
    assert (pl > 0).sum() > 300
    assert np.allclose(m.mean(2), pl, rtol=5e-6, atol=1e-300)


def _tri_average(fn, V, T, m=24):
    """Averages of fn(P) [.., 3] over each triangle by the midpoint rule on m^2
    sub-triangles (barycentric centroids)."""
    pts = []
    for i in range(m):
        for j in range(m - i):
            pts.append(((i + 1 / 3) / m, (j + 1 / 3) / m))        # upright sub-triangles
            if i + j < m - 1:
                pts.append(((i + 2 / 3) / m, (j + 2 / 3) / m))    # inverted ones
    b = np.array(pts)
    out = np.empty(len(T))
    for k, t in enumerate(T):
        a, bb, c = V[t].astype(np.float64)
        P = a + np.outer(b[:, 0], bb - a) + np.outer(b[:, 1], c - a)
        out[k] = fn(P).mean()
    return out


def test_tilted_mesh_free_space_closed_form(orc):
    """Free space over a tilted, ragged mesh: each triangle's value is the
    triangle average of Friis' (lambda / 4 pi d)^2 within 3 / sqrt(n_i), n_i the
    expected number of lattice rays through the triangle (n_i >= 100).  A wrong
    area, or the plane's |k_z| in place of the triangle's |n . k|, fails it."""
    sc = S.empty_scene()
    f = 3.5e9
    lam = C0 / f
    N = 2_000_000
    src = np.array([0.3, -0.2, 10.0])
    tx = S.Tx(pos=tuple(src), num_rays=N)
    p = S.TraceParams(f, 0)
    rng = np.random.default_rng(3)
    V, T = grid_surface(-16.0, -16.0, 4.0, 8, 8, lambda X, Y: 1.5 + 0.25 * X - 0.15 * Y)
    V[:, :2] += rng.uniform(-0.8, 0.8, (len(V), 2)).astype(np.float32)   # ragged triangles
    V[:, 2] += rng.uniform(-0.5, 0.5, len(V)).astype(np.float32)
    m = orc.radio_map_mesh(sc, tx, p, V, T)["map"]
    gain = _tri_average(lambda P: (lam / (4 * math.pi)) ** 2 / ((P - src) ** 2).sum(1), V, T)
    areas, normals = [], []
    for t in T:
        a, b, c = V[t].astype(np.float64)
        cr = np.cross(b - a, c - a)
        areas.append(0.5 * np.linalg.norm(cr))
        normals.append(cr / np.linalg.norm(cr))
    areas, normals = np.array(areas), np.array(normals)
    n_i = np.array([N / (4 * math.pi) * areas[k] * _tri_average(
        lambda P: np.abs((P - src) @ normals[k]) / np.linalg.norm(P - src, axis=1) ** 3, V, T[k:k + 1])[0]
        for k in range(len(T))])
    ok = n_i >= 100
    assert ok.sum() > 100
    rel = np.abs(m / gain - 1)
    assert np.all(rel[ok] <= 3 / np.sqrt(n_i[ok])), rel[ok].max()


def test_mesh_replay_of_own_record_and_slack(orc):
    """Replay of the oracle's own record reproduces the mesh map exactly with no
    adoption, and a crossing that lands on a shared vertex (the TX straight
    above a grid vertex: the south-pole lattice ray) is counted in every
    triangle sharing it and reported in their slack."""
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride, tx.ray_count = 4999, 2000
    V, T = grid_surface(-64.0, -64.0, 4.0, 32, 32, lambda X, Y: 1.5 + 0.5 * np.sin(X / 9.0) * np.cos(Y / 7.0))
    a = orc.radio_map_mesh(sc, tx, p, V, T, want_record=True)
    b = orc.radio_map_mesh(sc, tx, p, V, T, mode="replay", record=a["record"])
    rep = b["report"]
    assert rep["failures"] == 0 and rep["adopted_hit"] == rep["adopted_decision"] == 0
    assert rep["deposits"] > 500
    assert np.array_equal(a["map"], b["map"])
    # vertex hit: the pole ray of an N = 2 lattice points straight down
    one = S.Tx(pos=(0.0, 0.0, 10.0), num_rays=2, ray_begin=1, ray_count=1)
    Vf, Tf = grid_surface(-4.0, -4.0, 2.0, 4, 4, flat(1.5))
    e = S.empty_scene()
    r = orc.radio_map_mesh(e, one, S.TraceParams(3.5e9, 0), Vf, Tf, slack=True)
    hit = np.flatnonzero(r["map"] > 0)
    assert len(hit) >= 2                                   # every triangle sharing the vertex
    assert np.all(r["slack"][hit] >= r["map"][hit])


def test_mesh_gradient_equals_planar_gradient(orc):
    """Dual-number gradient on a flat mesh that tiles the planar cells, with
    each triangle weighted by half its cell's dL/dC: sum_i g_i C_i equals the
    planar functional (the pair mean is the cell), so the material gradients
    agree (to the FP32-area rounding of the mesh), and both TX-position
    gradients of box cells vanish."""
    sc, txs, p = S.workload(4)
    tx = txs[0]
    tx.ray_stride = 53
    p.deposit = 0
    p.nx = p.ny = 64            # 8192 surface triangles: the oracle tests each one per segment
    p.cell_size *= 4
    x0, y0 = p.map_corner()
    V, T = grid_surface(x0, y0, p.cell_size, p.nx, p.ny, flat(p.map_origin[2]))
    g = np.random.default_rng(5).uniform(0.0, 1.0, (p.ny, p.nx))
    rec = orc.radio_map(sc, tx, p, want_record=True)["record"]
    de, ds, dt = orc.grad(sc, tx, p, rec, g)
    gm = np.repeat(g.ravel() / 2.0, 2)
    rec_m = orc.radio_map_mesh(sc, tx, p, V, T, want_record=True)["record"]
    assert np.array_equal(rec_m[..., 0], rec[..., 0]) and np.array_equal(rec_m[..., 3], rec[..., 3])
    me, ms, mt = orc.grad_mesh(sc, tx, p, V, T, rec_m, gm)
    ref = np.concatenate([de, ds])
    assert np.abs(ref).max() > 0
    assert np.allclose(np.concatenate([me, ms]), ref, rtol=2e-5, atol=2e-5 * np.abs(ref).max())
    assert np.all(dt == 0.0) and np.all(mt == 0.0)


@pytest.mark.parametrize("ground", [None, 500.0])
def test_flat_mesh_diffraction_equals_planar_diffraction(orc, ground):
    """The diffraction map on a flat mesh that tiles the planar cells: each
    visible crossing falls into one triangle of its cell, the weighting factor
    on the triangle's plane equals the plane's, and 1/A is twice 1/cell^2, so
    the mean of a triangle pair equals the planar cell (FP32 vertices: 5e-6)."""
    sc = S.single_box(0.0, 20.0, 0.0, 30.0, 25.0, mat=(5.0, 0.1, 0.2), ground=ground)
    p = S.TraceParams(3.5e9, 0, cell_size=4.0, nx=20, ny=20, map_origin=(10.3, 15.2, 1.5))
    tx = S.Tx(pos=(-30.0, -20.0, 15.0), num_rays=1)
    x0, y0 = p.map_corner()
    V, T = grid_surface(x0, y0, p.cell_size, p.nx, p.ny, flat(p.map_origin[2]))
    pl = orc.diffraction_map(sc, tx, p, 512)["map"]
    m = orc.diffraction_map_mesh(sc, tx, p, 512, V, T)["map"].reshape(p.ny, p.nx, 2)
    assert (pl > 0).sum() > 100
    assert np.allclose(m.mean(2), pl, rtol=5e-6, atol=1e-300)


def test_mesh_diffraction_replay_of_own_record(orc):
    sc = S.single_box(0.0, 20.0, 0.0, 30.0, 25.0, mat=(5.0, 0.1, 0.2), ground=500.0)
    p = S.TraceParams(3.5e9, 0)
    tx = S.Tx(pos=(-30.0, -20.0, 15.0), num_rays=1)
    V, T = grid_surface(-40.0, -40.0, 5.0, 20, 20, lambda X, Y: 1.5 + 0.4 * np.sin(X / 6.0))
    a = orc.diffraction_map_mesh(sc, tx, p, 256, V, T, want_record=True)
    b = orc.diffraction_map_mesh(sc, tx, p, 256, V, T, mode="replay", record=a["record"], slack=True)
    assert b["report"]["failures"] == 0 and b["report"]["adopted_hit"] == 0
    assert np.array_equal(a["map"], b["map"])
    assert (a["map"] > 0).sum() > 50 and np.all(b["slack"] >= 0)
