"""GPU parity of diffuse reflection (App. A.10; sampling Eq.
path-solver-used-dist-event; a new tube per diffuse point in the estimator of
Sec. 4): forward maps replay-checked against the FP64 oracle, and the adjoint
against the oracle's dual numbers."""
import copy

import numpy as np
import pytest
import torch

from synth import scenes as S
from gpu_helpers import compare_maps, coin

pytestmark = pytest.mark.gpu
GRAD_RTOL = 1e-2


def _diffuse(sc, S_=(0.3, 0.5, 0.7, 0.4), pattern=(0, 1, 2, 0)):
    nm = sc.nm
    s = np.resize(np.asarray(S_, float), nm)
    pat = np.resize(np.asarray(pattern), nm)
    return sc.with_scattering(s, 0.2, pat, 3, 2, 0.6)


def _manhattan(stride=97):
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = stride
    p.diffuse = True
    return _diffuse(sc), tx, p


def _run(api, sc, tx, p, builder="auto"):
    gs = api.Scene.from_obj(sc, builder=builder)
    r = api.trace(gs, [tx], coin(p), record=True)
    torch.cuda.synchronize()
    out = (r["maps"][0].cpu().numpy(), r["record"].cpu().numpy(), r["stats"])
    gs.free()
    return out


@pytest.mark.parametrize("builder", ["auto", "sah"])
def test_diffuse_map_parity(orc, api, builder):
    """builder "sah": the diffuse tracer's single-site traversal on the binned-SAH tree."""
    sc, tx, p = _manhattan()
    m, rec, st = _run(api, sc, tx, p, builder)
    dec = rec[:, 3]
    assert ((dec >= 0) & (dec & 3 == 2)).sum() > 1000
    compare_maps(orc, sc, tx, p, m, rec)


@pytest.mark.parametrize("pol,deposit", [(2, 0), (0, 1)])
def test_diffuse_dual_pol_and_bilinear(orc, api, pol, deposit):
    sc, tx, p = _manhattan(stride=211)
    tx.pol = pol
    tx.pattern = 1
    p.deposit = deposit
    sc = _diffuse(sc, S_=(0.6, 0.8, 0.5, 0.9), pattern=(2, 0, 1, 2))
    m, rec, _ = _run(api, sc, tx, p)
    compare_maps(orc, sc, tx, p, m, rec)


def test_diffuse_with_early_termination(orc, api):
    sc, tx, p = _manhattan(stride=149)
    p.rr_depth, p.rr_max_prob, p.gain_threshold = 2, 0.5, 1e-13
    m, rec, _ = _run(api, sc, tx, p)
    dec = rec[:, 3]
    assert ((dec >= 0) & ((dec & 12) != 0)).sum() > 0
    compare_maps(orc, sc, tx, p, m, rec)


def test_diffuse_flag_off_is_specular(api):
    sc, tx, p = _manhattan(stride=997)
    p0 = copy.copy(p)
    p0.diffuse = False
    a, _, _ = _run(api, sc, tx, p0)
    b, _, _ = _run(api, S.workload(2)[0], tx, p0)
    assert np.array_equal(a, b)


def _grad_setup(stride=13, deposit=1):
    sc, txs, p = S.workload(4)
    sc = sc.with_scattering(np.linspace(0.2, 0.8, sc.nm), 0.3, np.arange(sc.nm) % 3, 2, 3, 0.5)
    tx = txs[0]
    tx.ray_stride = stride
    p.deposit = deposit
    p.diffuse = True
    return sc, tx, p


def test_diffuse_adjoint_retrace_takes_forward_choices(api):
    sc, tx, p = _grad_setup()
    gs = api.Scene.from_obj(sc)
    f = api.trace(gs, [tx], p, record=True)
    a = api.grad(gs, [tx], p, torch.rand_like(f["maps"]), record=True)
    assert torch.equal(f["record"], a["record"])
    gs.free()


@pytest.mark.parametrize("deposit", [1, 0])
def test_diffuse_adjoint_matches_oracle_gradient(orc, api, deposit):
    sc, tx, p = _grad_setup(deposit=deposit)
    gs = api.Scene.from_obj(sc)
    f = api.trace(gs, [tx], p, record=True)
    rng = np.random.default_rng(5)
    g = torch.tensor(rng.normal(size=(1, p.ny, p.nx)), dtype=torch.float32, device="cuda")
    a = api.grad(gs, [tx], p, g)
    ad = np.concatenate([a["d_eps"].cpu().numpy(), a["d_sigma"].cpu().numpy(), a["d_tx"][0].cpu().numpy()])
    rec = f["record"].view(tx.count(), p.max_depth + 1, 4).cpu().numpy()
    assert ((rec[:, :, 3] >= 0) & (rec[:, :, 3] & 3 == 2)).sum() > 1000
    compare_maps(orc, sc, tx, p, f["maps"][0].cpu().numpy(), rec)
    de, ds, dt = orc.grad(sc, tx, p, rec, g[0].double().cpu().numpy())
    ref = np.concatenate([de, ds, dt])
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    err = np.abs(ad - ref) / scale
    assert np.all(err <= GRAD_RTOL), err
    if deposit == 0:
        assert np.all(ad[-3:] == 0.0)
    gs.free()


def test_diffuse_city_sampled(orc, api):
    """The largest scene with diffuse reflection on every material: a sampled
    lattice subset of one transmitter (every 333331st of its 1e8 rays, depth 8,
    2048 x 2048 map) through the 0.97M-triangle city's binned-SAH tree,
    replayed by the oracle (brute force over every triangle)."""
    sc, txs, p = S.workload(5)
    sc = _diffuse(sc)
    p.diffuse = True
    tx = copy.copy(txs[0])
    tx.ray_stride, tx.ray_begin = 333_331, 7
    m, rec, st = _run(api, sc, tx, p)
    dec = rec[:, 3]
    assert ((dec >= 0) & (dec & 3 == 2)).sum() > 40
    info = compare_maps(orc, sc, tx, p, m, rec)
    assert info["cells"] > 100


def test_diffuse_city_adjoint_matches_oracle(orc, api):
    """The adjoint with diffuse reflection on the largest scene: a sampled
    lattice subset of one city transmitter (depth 8, bilinear cells, 0.97M
    triangles), gradient of sum(g C) for a seeded g over the 2048 x 2048 map
    against the oracle's dual numbers along the GPU's record (which the oracle
    certifies first), the re-trace taking the forward's choices."""
    sc, txs, p = S.workload(5)
    sc = _diffuse(sc)
    p.diffuse = True
    p.deposit = 1
    tx = copy.copy(txs[0])
    tx.ray_stride, tx.ray_begin = 333_331, 7
    gs = api.Scene.from_obj(sc)
    f = api.trace(gs, [tx], p, record=True)
    g = torch.tensor(np.random.default_rng(9).normal(size=(1, p.ny, p.nx)), dtype=torch.float32, device="cuda")
    a = api.grad(gs, [tx], p, g, record=True)
    assert torch.equal(f["record"], a["record"])
    ad = np.concatenate([a["d_eps"].cpu().numpy(), a["d_sigma"].cpu().numpy(), a["d_tx"][0].cpu().numpy()])
    rec = f["record"].view(tx.count(), p.max_depth + 1, 4).cpu().numpy()
    assert ((rec[:, :, 3] >= 0) & (rec[:, :, 3] & 3 == 2)).sum() > 40
    compare_maps(orc, sc, tx, p, f["maps"][0].cpu().numpy(), rec)
    de, ds, dt = orc.grad(sc, tx, p, rec, g[0].double().cpu().numpy())
    ref = np.concatenate([de, ds, dt])
    assert np.abs(ref[:2 * sc.nm]).max() > 0
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    err = np.abs(ad - ref) / scale
    assert np.all(err <= GRAD_RTOL), err
    gs.free()
