"""GPU parity of the 'next' rows: synthetic transmit arrays (Sec. 4.4) and
early termination by gain thresholding and Russian roulette (Sec. 4.5)."""
import copy

import numpy as np
import pytest
import torch

from synth import scenes as S
from gpu_helpers import compare_maps, coin

pytestmark = pytest.mark.gpu


def _manhattan(stride=97):
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = stride
    return sc, tx, p


def _run(api, sc, tx, p):
    gs = api.Scene.from_obj(sc)
    r = api.trace(gs, [tx], coin(p), record=True)
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
    info = compare_maps(orc, sc, tx, p, m, rec)
    assert info["frac_within_rtol"] >= 0.999, info


@pytest.mark.parametrize("nant", [1, 2, 17, 37, 64])
def test_array_sizes(orc, api, nant):
    """Edge and ragged sizes of the array-factor paths: one element (per-element
    path), two (a uniform linear array of one short block), 17 (one block plus a
    ragged one), 37 (a pair of 16-element blocks plus a ragged block) and 64 (two
    pairs), steered precoding along an oblique axis."""
    sc, tx, p = _manhattan(stride=211)
    lam = 299792458.0 / p.freq_hz
    axis = np.array([0.6, -0.3, 0.74])
    axis /= np.linalg.norm(axis)
    tx.ant_pos = np.outer(np.arange(nant) - 0.5 * (nant - 1), axis) * 0.5 * lam
    k = np.array([0.2, 0.9, -0.4]) / np.linalg.norm([0.2, 0.9, -0.4])
    w = np.exp(-2j * np.pi / lam * (tx.ant_pos @ k)) / np.sqrt(nant)
    tx.precoding = w
    m, rec, _ = _run(api, sc, tx, p)
    info = compare_maps(orc, sc, tx, p, m, rec)
    assert info["frac_within_rtol"] >= 0.999, info


def test_irregular_array(orc, api):
    """Elements off any regular line (the per-element path): 48 seeded positions
    in a 2 m x 0.3 m x 0.3 m box (phases up to ~600 rad at 28 GHz) with seeded
    complex precoding."""
    sc, tx, p = _manhattan(stride=89)
    rng = np.random.default_rng(12)
    tx.ant_pos = rng.uniform(-1.0, 1.0, size=(48, 3)) * np.array([1.0, 0.15, 0.15])
    w = rng.normal(size=48) + 1j * rng.normal(size=48)
    tx.precoding = w / np.linalg.norm(w)
    m, rec, _ = _run(api, sc, tx, p)
    info = compare_maps(orc, sc, tx, p, m, rec)
    assert info["frac_within_rtol"] >= 0.99, info


def test_street_canyon_1024_element_array(orc, api):
    """The largest array of the time-vs-N_S-and-N_A study (Sec. 4.4): a
    1024-element half-wavelength ULA 20 m above a street canyon, depth 5, on a
    lattice subset of a 1e8-sample launch.  Phases reach k0 |d| ~ 1600 rad and
    a ray near a null of the array factor has no FP32 answer within 1e-3, so
    every cell is held to 1e-3 plus the oracle's worst-case bound on the
    double-float array factor, and 99 % of the cells to 1e-3 alone."""
    sc = S.street_canyon()
    p = S.TraceParams(3.5e9, 5, cell_size=1.0, nx=256, ny=256)
    tx = S.Tx(pos=(0.0, 0.0, 20.0), num_rays=100_000_000, seed=11)
    tx.ray_stride, tx.ray_begin = 20_011, 5
    tx.ant_pos, tx.precoding = S.uniform_linear_array(1024, p.freq_hz, 0.5)
    m, rec, st = _run(api, sc, tx, p)
    assert st["rays"] == tx.count()
    info = compare_maps(orc, sc, tx, p, m, rec)
    assert info["cells"] > 500
    assert info["frac_within_rtol"] >= 0.99, info


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


def test_city_roulette_array_dual_pol(orc, api):
    """The largest scene with the widened model at once: Russian roulette after
    two interactions (p_max = 0.5), a steered 16-element uniform linear array and
    dual polarisation, on a sampled lattice subset of one city transmitter
    (depth 8, 0.97M triangles, binned-SAH tree), replayed by the oracle."""
    sc, txs, p = S.workload(5)
    tx = copy.copy(txs[0])
    tx.ray_stride, tx.ray_begin = 166_661, 7
    tx.pol = 2
    tx.ant_pos, tx.precoding = S.uniform_linear_array(16, p.freq_hz, 0.5, axis=1, steer=(0.3, 1.0, -0.2))
    p.rr_depth, p.rr_max_prob, p.gain_threshold = 2, 0.5, 0.0
    m, rec, st = _run(api, sc, tx, p)
    dec = rec[:, 3]
    assert int(((dec >= 0) & ((dec & 12) != 0)).sum()) > 100      # roulette kills
    info = compare_maps(orc, sc, tx, p, m, rec)
    assert info["cells"] > 100
    assert info["frac_within_rtol"] >= 0.99, info


def test_array_factor_prepass_equals_inline(api):
    """The array factor that trace and gradient calls take from the pre-pass
    kernel (four unrolled Horner chains) equals, bit for bit, the tracer's
    inline form (two rolled chains; graph plans and the no-allocation entry
    point), for every work item of one call mixing a 1024-element and a
    37-element (ragged) steered uniform linear array, a 48-element irregular
    array and a transmitter without an array (whose entries stay unwritten)."""
    import ctypes as C
    from paper_2504_21719_b300 import _lib as L
    sc, txs, p = S.workload(2)
    base = txs[0]
    tl = []
    for k, (na, steer) in enumerate([(1024, (0.3, 1.0, -0.2)), (37, (1.0, 0.2, 0.1)), (48, None), (0, None)]):
        t = copy.copy(base)
        t.ray_stride, t.ray_begin = 97 + 2 * k, k
        t.yaw = 0.3 * k
        if na and steer is not None:
            t.ant_pos, t.precoding = S.uniform_linear_array(na, p.freq_hz, 0.5, axis=k % 3, steer=steer)
        elif na:
            rng = np.random.default_rng(12)
            t.ant_pos = rng.uniform(-1.0, 1.0, size=(na, 3)) * np.array([1.0, 0.15, 0.15])
            w = rng.normal(size=na) + 1j * rng.normal(size=na)
            t.precoding = w / np.linalg.norm(w)
        tl.append(t)
    gs = api.Scene.from_obj(sc)
    arr, ntx = api._tx_array(tl)
    prm = api.params_from(p)
    total = sum(t.count() for t in tl)
    a = torch.full((total, 2), float("nan"), dtype=torch.float32, device="cuda")
    b = torch.full((total, 2), float("nan"), dtype=torch.float32, device="cuda")
    lib = L.load()
    rc = lib.rm_debug_array_factor(gs.handle, arr, ntx, C.byref(prm), C.c_void_p(a.data_ptr()),
                                   C.c_void_p(b.data_ptr()), total, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.RM_OK, lib.rm_last_error()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    n_arr = sum(t.count() for t in tl[:3])
    assert torch.isfinite(a[:n_arr]).all() and torch.isnan(a[n_arr:]).all()
    assert (a[:n_arr].abs().sum(1) > 0).all()
    rc = lib.rm_debug_array_factor(gs.handle, arr, ntx, C.byref(prm), C.c_void_p(a.data_ptr()),
                                   C.c_void_p(b.data_ptr()), total - 1, None)
    assert rc == L.RM_EINVAL
    gs.free()


def test_array_above_prepass_limit_matches_halves(api):
    """A call of more than 2^31 rays with a synthetic array evaluates the array
    factor at each ray's launch instead of in the pre-pass (whose buffer holds
    at most 2^31 rays); its map equals the sum of the maps of its two lattice
    halves, each of which takes the pre-pass (depth 0 over a ground plane)."""
    sc = S.ground_plane(500.0)
    p = S.TraceParams(3.5e9, 0, reflect=False, refract=False, cell_size=10.0, nx=100, ny=100)
    tx = S.Tx(pos=(0.0, 0.0, 10.0), num_rays=2 ** 31 + 1000, seed=5)
    tx.ant_pos, tx.precoding = S.uniform_linear_array(16, p.freq_hz, 0.5, axis=0, steer=(0.4, 0.2, -0.9))
    gs = api.Scene.from_obj(sc)
    full = api.trace(gs, [tx], p)
    assert full["stats"]["rays"] == tx.num_rays
    parts = torch.zeros_like(full["maps"], dtype=torch.float64)
    for b in range(2):
        h = copy.copy(tx)
        h.ray_begin, h.ray_stride = b, 2
        parts += api.trace(gs, [h], p)["maps"].double()
    fm = full["maps"].double()
    mask = fm > 1e-15
    assert mask.sum() > 5000
    assert torch.all((parts - fm).abs()[mask] <= 2e-5 * fm[mask])
    gs.free()
