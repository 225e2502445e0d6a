"""Seeded synthetic scenes and transmitter sets for SBR radio maps.

This module only generates inputs: meshes, per-triangle material ids, the
material table {relative permittivity, conductivity, slab thickness} and
transmitter placements.  It holds none of the method's arithmetic (no
permittivity, Fresnel or ray math), so both the FP64 CPU oracle and the CUDA
path can consume exactly the same FP32 vertices.

A scene follows the paper's mesh model (Sec. 2.1): a set of triangles, each
triangle carrying the index of its radio material.  Objects are flattened into
one global triangle array; the ground plane, when present, always holds
triangle indices 0 and 1.

All random draws use ``numpy.random.Generator(PCG64(seed))`` in the order
written in each function, so a scene is a pure function of its seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Ground material used throughout: permittivity 5.24, conductivity 0.0462 S/m,
# modelled as a half-space (thickness <= 0 means no transmission).
GROUND = (5.24, 0.0462, 0.0)
# Building walls are single-layer slabs of this thickness (m).
WALL_THICKNESS = 0.2


@dataclass
class Scene:
    name: str
    verts: np.ndarray      # float32 [nv, 3]
    tris: np.ndarray       # int32 [nt, 3]
    tri_mat: np.ndarray    # int32 [nt]
    mats: np.ndarray       # float32 [nm, 3] = (eps_r, sigma S/m, thickness m)
    footprints: list = field(default_factory=list)  # (cx, cy, r) or (x0,x1,y0,y1)
    # diffuse reflection parameters, float32 [nm, 6] = (S, K_x, pattern, alpha_R,
    # alpha_I, Lambda) with pattern 0 Lambertian, 1 directive, 2 backscattering;
    # None = no diffuse reflection (S = 0)
    scat: np.ndarray | None = None

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])

    @property
    def nm(self) -> int:
        return int(self.mats.shape[0])

    def save(self, path: str) -> None:
        extra = {} if self.scat is None else {"scat": self.scat}
        np.savez(path, verts=self.verts, tris=self.tris, tri_mat=self.tri_mat,
                 mats=self.mats, name=np.array(self.name), **extra)

    @staticmethod
    def load(path: str) -> "Scene":
        z = np.load(path)
        return Scene(str(z["name"]), z["verts"], z["tris"], z["tri_mat"], z["mats"],
                     scat=z["scat"] if "scat" in z else None)

    def with_scattering(self, S, K_x=0.0, pattern=0, alpha_r=1, alpha_i=1, lam=1.0) -> "Scene":
        """A copy whose materials all get the diffuse parameters given (scalars or
        per-material sequences)."""
        nm = self.nm
        cols = [np.broadcast_to(np.asarray(c, np.float32), (nm,)) for c in (S, K_x, pattern, alpha_r, alpha_i, lam)]
        return Scene(self.name, self.verts, self.tris, self.tri_mat, self.mats, list(self.footprints),
                     np.ascontiguousarray(np.stack(cols, 1)))


@dataclass
class Tx:
    """One transmitter: position, yaw/pitch/roll (rad), antenna and lattice subset."""
    pos: tuple
    num_rays: int
    yaw: float = 0.0
    pitch: float = 0.0
    roll: float = 0.0
    pol: int = 0          # 0 = vertical (theta), 1 = horizontal (phi), 2 = dual
    pattern: int = 0      # 0 = isotropic, 1 = short dipole
    ray_begin: int = 0
    ray_count: int = -1   # -1 = all num_rays
    ray_stride: int = 1
    seed: int = 0
    ant_pos: object = None      # synthetic array: [n_ant, 3] element positions (m), antenna frame
    precoding: object = None    # [n_ant] complex precoding weights

    def count(self) -> int:
        if self.ray_count >= 0:
            return self.ray_count
        return (self.num_rays - self.ray_begin + self.ray_stride - 1) // self.ray_stride


@dataclass
class TraceParams:
    freq_hz: float
    max_depth: int
    reflect: bool = True
    refract: bool = True
    los: bool = True
    map_origin: tuple = (0.0, 0.0, 1.5)   # centre of the map, plane z = origin[2]
    cell_size: float = 1.0
    nx: int = 100
    ny: int = 100
    deposit: int = 0      # 0 = box cells, 1 = bilinear (tent) splat
    rr_depth: int = 0     # early termination after this many interactions (0 = off)
    rr_max_prob: float = 0.0
    gain_threshold: float = 0.0
    diffuse: bool = False  # diffuse reflection on materials with S > 0

    def map_corner(self):
        """Lower-left corner (x0, y0) of a map centred on map_origin."""
        return (self.map_origin[0] - 0.5 * self.nx * self.cell_size,
                self.map_origin[1] - 0.5 * self.ny * self.cell_size)


# ----------------------------------------------------------------------------
# mesh helpers
# ----------------------------------------------------------------------------

def _quad_ground(half: float, z: float = 0.0):
    v = np.array([[-half, -half, z], [half, -half, z], [half, half, z], [-half, half, z]],
                 dtype=np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return v, t


def _box(x0, x1, y0, y1, z0, z1):
    """8 corners and 12 outward-wound triangles of an axis-aligned box."""
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float32)
    t = np.array([
        [0, 2, 1], [0, 3, 2],      # bottom (-z)
        [4, 5, 6], [4, 6, 7],      # top (+z)
        [0, 1, 5], [0, 5, 4],      # -y
        [2, 3, 7], [2, 7, 6],      # +y
        [1, 2, 6], [1, 6, 5],      # +x
        [3, 0, 4], [3, 4, 7],      # -x
    ], dtype=np.int32)
    return v, t


class _MeshBuilder:
    def __init__(self):
        self.v, self.t, self.m = [], [], []
        self.nv = 0

    def add(self, verts, tris, mat):
        self.v.append(np.asarray(verts, np.float32))
        self.t.append(np.asarray(tris, np.int32) + self.nv)
        self.m.append(np.full(len(tris), mat, np.int32))
        self.nv += len(verts)

    def build(self):
        if not self.v:
            return (np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32),
                    np.zeros((0,), np.int32))
        return (np.concatenate(self.v), np.concatenate(self.t), np.concatenate(self.m))


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def empty_scene() -> Scene:
    return Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32),
                 np.zeros((0,), np.int32), np.array([GROUND], np.float32))


def ground_plane(half: float = 500.0, mat=GROUND) -> Scene:
    """Two triangles covering [-half, half]^2 at z = 0 (1 km square by default)."""
    v, t = _quad_ground(half)
    return Scene("ground", v, t, np.zeros(2, np.int32), np.array([mat], np.float32))


def manhattan(seed: int = 2, n_building_mats: int = 3, nblocks: int = 10,
              footprint: float = 40.0, street: float = 20.0, hmin: float = 10.0,
              hmax: float = 60.0, ground_half: float = 500.0) -> Scene:
    """Manhattan grid of box buildings (12 triangles each) on a ground plane.

    Block pitch = footprint + street; the grid is centred so that (0, 0) is a
    street intersection.  Draw order: heights U(hmin, hmax) per building,
    permittivities U(3, 7) and conductivities 10^U(-3, 0) per building
    material, then the material index of each building, uniform over
    1..n_building_mats.  Material 0 is the ground half-space.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = nblocks * nblocks
    heights = rng.uniform(hmin, hmax, size=nb)
    eps = rng.uniform(3.0, 7.0, size=n_building_mats)
    sig = 10.0 ** rng.uniform(-3.0, 0.0, size=n_building_mats)
    bmat = rng.integers(1, n_building_mats + 1, size=nb)

    mats = [GROUND] + [(float(e), float(s), WALL_THICKNESS) for e, s in zip(eps, sig)]
    mb = _MeshBuilder()
    gv, gt = _quad_ground(ground_half)
    mb.add(gv, gt, 0)
    pitch = footprint + street
    c0 = -0.5 * pitch * (nblocks - 1)
    fps = []
    for j in range(nblocks):
        for i in range(nblocks):
            b = j * nblocks + i
            cx, cy = c0 + i * pitch, c0 + j * pitch
            x0, x1 = cx - 0.5 * footprint, cx + 0.5 * footprint
            y0, y1 = cy - 0.5 * footprint, cy + 0.5 * footprint
            bv, bt = _box(x0, x1, y0, y1, 0.0, float(heights[b]))
            mb.add(bv, bt, int(bmat[b]))
            fps.append((x0, x1, y0, y1))
    v, t, m = mb.build()
    return Scene(f"manhattan(seed={seed},nm={n_building_mats + 1})", v, t, m,
                 np.array(mats, np.float32), fps)


def street_canyon(seed: int = 7, per_side: int = 6, length: float = 30.0, gap: float = 10.0,
                  depth: float = 20.0, street: float = 20.0, hmin: float = 15.0, hmax: float = 40.0,
                  ground_half: float = 300.0) -> Scene:
    """A straight street along x (width `street`, centred on y = 0) lined on each
    side by `per_side` box buildings of `length` x `depth` m with `gap` m between
    them, on a ground plane: a seeded stand-in for a small street-canyon scene.

    Draw order: heights U(hmin, hmax), south row then north row, west to east.
    Material 0 is the ground half-space, material 1 the building walls."""
    rng = np.random.Generator(np.random.PCG64(seed))
    heights = rng.uniform(hmin, hmax, size=2 * per_side)
    mats = [GROUND, (5.24, 0.123, WALL_THICKNESS)]
    mb = _MeshBuilder()
    gv, gt = _quad_ground(ground_half)
    mb.add(gv, gt, 0)
    span = per_side * length + (per_side - 1) * gap
    fps = []
    for row, (y0, y1) in enumerate([(-0.5 * street - depth, -0.5 * street), (0.5 * street, 0.5 * street + depth)]):
        for i in range(per_side):
            x0 = -0.5 * span + i * (length + gap)
            bv, bt = _box(x0, x0 + length, y0, y1, 0.0, float(heights[row * per_side + i]))
            mb.add(bv, bt, 1)
            fps.append((x0, x0 + length, y0, y1))
    v, t, m = mb.build()
    return Scene(f"street_canyon(seed={seed})", v, t, m, np.array(mats, np.float32), fps)


def procedural_city(seed: int = 5, ncells: int = 210, cell: float = 19.0,
                    jitter: float = 1.5, nmin: int = 4, nmax: int = 12,
                    rmin: float = 4.0, rmax: float = 8.0, h_median: float = 20.0,
                    h_sigma_ln: float = 0.5, n_building_mats: int = 7,
                    ground_half: float = 2000.0) -> Scene:
    """City of extruded convex n-gons on a grid (about 1M triangles at defaults).

    Each grid cell holds one building: a polygon with n ~ U{nmin..nmax}
    vertices at sorted random angles on a circle of radius U(rmin, rmax) around
    the jittered cell centre (inscribed, hence convex; rmax + jitter <= cell/2,
    hence no overlaps), extruded to a log-normal height.  A building has n - 2
    roof triangles and 2n wall triangles (no floor).  Draw order: jitter x,
    jitter y, n, radius, height, material id per building (vectorised), then
    the sorted angles per building in row-major cell order, then the building
    material table.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = ncells * ncells
    jx = rng.uniform(-jitter, jitter, size=nb)
    jy = rng.uniform(-jitter, jitter, size=nb)
    nv = rng.integers(nmin, nmax + 1, size=nb)
    rad = rng.uniform(rmin, rmax, size=nb)
    hgt = np.exp(math.log(h_median) + h_sigma_ln * rng.standard_normal(size=nb))
    bmat = rng.integers(1, n_building_mats + 1, size=nb)
    ang = [np.sort(rng.uniform(0.0, 2.0 * math.pi, size=int(k))) for k in nv]
    eps = rng.uniform(3.0, 7.0, size=n_building_mats)
    sig = 10.0 ** rng.uniform(-3.0, 0.0, size=n_building_mats)
    mats = [GROUND] + [(float(e), float(s), WALL_THICKNESS) for e, s in zip(eps, sig)]

    half = 0.5 * ncells * cell
    idx = np.arange(nb)
    cx = -half + cell * (idx % ncells + 0.5) + jx
    cy = -half + cell * (idx // ncells + 0.5) + jy

    gv, gt = _quad_ground(ground_half)
    vs, ts, ms = [gv], [gt], [np.zeros(2, np.int32)]
    base = 4
    for b in range(nb):
        k = int(nv[b])
        a = ang[b]
        px = cx[b] + rad[b] * np.cos(a)
        py = cy[b] + rad[b] * np.sin(a)
        bot = np.stack([px, py, np.zeros(k)], 1)
        top = np.stack([px, py, np.full(k, hgt[b])], 1)
        vs.append(np.concatenate([bot, top]).astype(np.float32))
        i = np.arange(k)
        j = (i + 1) % k
        walls = np.concatenate([np.stack([i, j, k + j], 1), np.stack([i, k + j, k + i], 1)])
        fan = np.stack([np.full(k - 2, k), k + np.arange(1, k - 1), k + np.arange(2, k)], 1)
        tri = np.concatenate([fan, walls]).astype(np.int32) + base
        ts.append(tri)
        ms.append(np.full(len(tri), bmat[b], np.int32))
        base += 2 * k
    fps = [(float(cx[b]), float(cy[b]), float(rad[b])) for b in range(nb)]
    return Scene(f"city(seed={seed})", np.concatenate(vs), np.concatenate(ts),
                 np.concatenate(ms), np.array(mats, np.float32), fps)


def single_wall(x: float = 20.0, half_w: float = 50.0, h: float = 40.0,
                mat=(4.0, 0.01, WALL_THICKNESS)) -> Scene:
    """One vertical wall in the plane x = const, material 0."""
    v = np.array([[x, -half_w, 0], [x, half_w, 0], [x, half_w, h], [x, -half_w, h]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return Scene("wall", v, t, np.zeros(2, np.int32), np.array([mat], np.float32))


def terrain_surface(half: float = 256.0, n: int = 256, z0: float = 1.5, amp: float = 0.5):
    """A measurement surface: an n x n grid of square cells over [-half, half]^2, two
    triangles per cell (cell (iy, ix) -> triangles 2 (iy n + ix) and the next), at the
    rolling height z0 + amp sin(x / 9) cos(y / 7).  Returns (verts f32 [(n+1)^2, 3],
    tris i32 [2 n^2, 3])."""
    xs = np.linspace(-half, half, n + 1)
    X, Y = np.meshgrid(xs, xs)
    V = np.stack([X.ravel(), Y.ravel(), (z0 + amp * np.sin(X / 9.0) * np.cos(Y / 7.0)).ravel()], 1)
    a = (np.arange(n)[:, None] * (n + 1) + np.arange(n)[None, :]).ravel()
    T = np.empty((2 * n * n, 3), np.int64)
    T[0::2] = np.stack([a, a + 1, a + n + 2], 1)
    T[1::2] = np.stack([a, a + n + 2, a + n + 1], 1)
    return V.astype(np.float32), T.astype(np.int32)


def ground_and_wall(ground_half: float = 500.0, x: float = 20.0, half_w: float = 100.0,
                    h: float = 60.0, wall_mat=(4.0, 0.01, 0.0)) -> Scene:
    """Ground (material 0, triangles 0-1) plus one wall at x = const (material 1)."""
    mb = _MeshBuilder()
    gv, gt = _quad_ground(ground_half)
    mb.add(gv, gt, 0)
    v = np.array([[x, -half_w, 0], [x, half_w, 0], [x, half_w, h], [x, -half_w, h]], np.float32)
    mb.add(v, np.array([[0, 1, 2], [0, 2, 3]], np.int32), 1)
    vv, tt, mm = mb.build()
    return Scene("ground+wall", vv, tt, mm, np.array([GROUND, wall_mat], np.float32))


def single_box(x0=0.0, x1=20.0, y0=0.0, y1=30.0, h=25.0, mat=(5.0, 0.1, WALL_THICKNESS), ground=None) -> Scene:
    """One box building [x0, x1] x [y0, y1] x [0, h] with outward-wound faces (12
    triangles, material 0), optionally on a square ground of half-size `ground`
    (material 1, half-space)."""
    mb = _MeshBuilder()
    if ground:
        gv, gt = _quad_ground(ground)
        mb.add(gv, gt, 1)
    v, t = _box(x0, x1, y0, y1, 0.0, h)
    mb.add(v, t, 0)
    vv, tt, mm = mb.build()
    mats = [mat] + ([GROUND] if ground else [])
    return Scene("single-box", vv, tt, mm, np.array(mats, np.float32))


def closed_box(half: float = 10.0, mat=(3.0, 0.0, WALL_THICKNESS)) -> Scene:
    """Closed box [-half, half]^3 of slab walls (lossless by default), 12 triangles."""
    v, t = _box(-half, half, -half, half, -half, half)
    return Scene("closed-box", v, t, np.zeros(12, np.int32), np.array([mat], np.float32))


def two_walls(gap: float = 30.0, half_w: float = 200.0, h: float = 200.0,
              mat=(5.0, 0.0, WALL_THICKNESS)) -> Scene:
    """Two parallel slab walls at x = +-gap/2 (a lossless 'corridor' without ground)."""
    mb = _MeshBuilder()
    for x in (-0.5 * gap, 0.5 * gap):
        v = np.array([[x, -half_w, -h], [x, half_w, -h], [x, half_w, h], [x, -half_w, h]],
                     np.float32)
        mb.add(v, np.array([[0, 1, 2], [0, 2, 3]], np.int32), 0)
    vv, tt, mm = mb.build()
    return Scene("two-walls", vv, tt, mm, np.array([mat], np.float32))


# ----------------------------------------------------------------------------
# transmitters and materials
# ----------------------------------------------------------------------------

def _inside_footprint(scene: Scene, x: float, y: float) -> bool:
    for fp in scene.footprints:
        if len(fp) == 4:
            x0, x1, y0, y1 = fp
            if x0 <= x <= x1 and y0 <= y <= y1:
                return True
        else:
            cx, cy, r = fp
            if (x - cx) ** 2 + (y - cy) ** 2 <= r * r:
                return True
    return False


def random_txs(scene: Scene, seed: int, n: int, half: float, hmin: float, hmax: float,
               log2_rays: tuple | None = None, num_rays: int | None = None):
    """n transmitters uniform in [-half, half]^2 outside every footprint.

    Draw order per transmitter: x, y (re-drawn while inside a footprint), then
    the height U(hmin, hmax); after all positions, the ray counts
    round(2^U(log2_rays)) when log2_rays is given.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        while True:
            x, y = rng.uniform(-half, half, size=2)
            if not _inside_footprint(scene, float(x), float(y)):
                break
        z = rng.uniform(hmin, hmax)
        out.append([float(x), float(y), float(z)])
    if log2_rays is not None:
        counts = np.rint(2.0 ** rng.uniform(log2_rays[0], log2_rays[1], size=n)).astype(np.int64)
    else:
        counts = np.full(n, int(num_rays), np.int64)
    return [Tx(pos=tuple(p), num_rays=int(c), seed=1000 + i) for i, (p, c) in enumerate(zip(out, counts))]


def city_transmitters(scene: Scene, n: int, num_rays: int = 100_000_000):
    """The city workload's transmitters (seed 50, heights U(10, 50) m, outside every
    footprint of the 3.8 km square), n of them: the first 16 of any n >= 16 are the
    workload's 16, so n = 16 N gives N disjoint 16-transmitter workloads."""
    return random_txs(scene, 50, n, 1900.0, 10.0, 50.0, num_rays=num_rays)


def perturb_materials(mats: np.ndarray, seed: int) -> np.ndarray:
    """Target materials: eps_r * (1 + 0.2 U(-1, 1)), sigma * exp(0.5 N(0, 1)).

    Draw order: all eps factors, then all sigma factors.  Thickness unchanged.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    m = np.array(mats, np.float64).copy()
    fe = 1.0 + 0.2 * rng.uniform(-1.0, 1.0, size=len(m))
    fs = np.exp(0.5 * rng.standard_normal(size=len(m)))
    m[:, 0] *= fe
    m[:, 1] *= fs
    return m.astype(np.float32)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def uniform_linear_array(n: int, freq_hz: float, spacing_wavelengths: float = 0.5, axis: int = 1,
                         steer=None):
    """Element positions of an n-element uniform linear array along a local axis
    and unit-norm precoding weights (uniform, or steering towards a direction).

    Positions only: no method arithmetic (the array factor is computed by the
    oracle and by the CUDA path, each on its own)."""
    lam = 299792458.0 / freq_hz
    pos = np.zeros((n, 3))
    pos[:, axis] = (np.arange(n) - 0.5 * (n - 1)) * spacing_wavelengths * lam
    w = np.ones(n, np.complex128) / np.sqrt(n)
    if steer is not None:
        k = np.asarray(steer, np.float64)
        k = k / np.linalg.norm(k)
        w = np.exp(-2j * np.pi / lam * (pos @ k)) / np.sqrt(n)
    return pos, w


def workload(cfg: int):
    """Return (scene, [Tx], TraceParams) for workload 1..5.

    1 two-ray ground plane, 3.5 GHz, 1e5 rays, depth 1, reflection only,
      100 x 100 cells of 2 m at z = 1.5 m.
    2 Manhattan (seed 2, 3 building materials), TX (0, 0, 30), 28 GHz, 1e7
      rays, depth 5, reflection + refraction, 512 x 512 cells of 1 m.
    3 same scene, 64 TX (seed 3) at heights U(5, 40) with 2^U(16, 22) rays,
      depth 3, 64 maps of 256 x 256 cells of 2 m.
    4 Manhattan (seed 4, 7 building materials), TX (0, 0, 30), 28 GHz, 1e6
      rays, depth 4, bilinear deposit, 256 x 256 cells of 2 m.
    5 procedural city (seed 5), 16 TX (seed 50), 1e8 rays each, depth 8,
      2048 x 2048 cells of 2 m.
    """
    if cfg == 1:
        sc = ground_plane(500.0)
        txs = [Tx(pos=(0.0, 0.0, 10.0), num_rays=100_000, seed=1)]
        p = TraceParams(3.5e9, 1, reflect=True, refract=False, cell_size=2.0, nx=100, ny=100)
        return sc, txs, p
    if cfg == 2:
        sc = manhattan(2, 3)
        txs = [Tx(pos=(0.0, 0.0, 30.0), num_rays=10_000_000, seed=2)]
        p = TraceParams(28e9, 5, cell_size=1.0, nx=512, ny=512)
        return sc, txs, p
    if cfg == 3:
        sc = manhattan(2, 3)
        txs = random_txs(sc, 3, 64, 300.0, 5.0, 40.0, log2_rays=(16.0, 22.0))
        p = TraceParams(28e9, 3, cell_size=2.0, nx=256, ny=256)
        return sc, txs, p
    if cfg == 4:
        sc = manhattan(4, 7)
        txs = [Tx(pos=(0.0, 0.0, 30.0), num_rays=1_000_000, seed=4)]
        p = TraceParams(28e9, 4, cell_size=2.0, nx=256, ny=256, deposit=1)
        return sc, txs, p
    if cfg == 5:
        sc = procedural_city(5)
        txs = city_transmitters(sc, 16)
        p = TraceParams(28e9, 8, cell_size=2.0, nx=2048, ny=2048)
        return sc, txs, p
    raise ValueError(f"unknown workload {cfg}")
