"""Pins of the oracle's diffuse reflection (App. A.10: Eqs. R, scattered_field,
lambertian_model, directive_model, backscattering_model; sampling Eq.
path-solver-used-dist-event; estimator weight 2 pi r^2 / |n.k_i| per diffuse
point, Eq. radio-map-solver-ci-all-2-estimator): scattering-pattern
normalisation by quadrature, the hemisphere sampler, the scattered field's
power and cross-polarisation split, energy bookkeeping in a lossless closed
box, the map of a Lambertian ground against a quadrature of the model's
integral, and the replay / frozen / gradient modes with diffuse events."""
import copy
import math

import numpy as np
import pytest

from synth import scenes as S

C0 = 299792458.0
EPS0 = 8.8541878128e-12


def _hemisphere_rule(n_t=96, n_p=192):
    """Directions and weights integrating over the upper (z >= 0) hemisphere:
    Gauss-Legendre in theta on [0, pi/2] (weight sin theta), trapezoid in phi."""
    g, w = np.polynomial.legendre.leggauss(n_t)
    th = (g + 1) * np.pi / 4
    wt = w * np.pi / 4 * np.sin(th)
    ph = np.arange(n_p) * 2 * np.pi / n_p
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    W = (wt[:, None] * np.full(n_p, 2 * np.pi / n_p)[None, :]).reshape(-1)
    return d, W


# ---------------------------------------------------------------------------
# scattering patterns
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pattern,aR,aI,lam", [(0, 1, 1, 1.0), (1, 1, 1, 1.0), (1, 2, 1, 1.0), (1, 5, 1, 1.0),
                                               (1, 12, 1, 1.0), (2, 3, 1, 0.6), (2, 8, 4, 0.25),
                                               (2, 2, 7, 0.0)])
def test_pattern_integrates_to_one(orc, pattern, aR, aI, lam):
    # the normalisation condition that accompanies Eq. scattered_field
    d, W = _hemisphere_rule()
    n = np.array([0.0, 0.0, 1.0])
    for th_i in (0.0, 0.3, 0.8, 1.2, 1.55):
        ki = np.array([math.sin(th_i), 0.0, -math.cos(th_i)])
        f = orc.scat_pattern(pattern, ki, n, d, aR, aI, lam)
        assert np.all(f >= 0.0)
        assert abs((f * W).sum() - 1.0) < 1e-9, (th_i, (f * W).sum())


def test_pattern_normalisation_on_tilted_surface(orc):
    # same condition for an arbitrary normal: rotate the rule onto n
    d, W = _hemisphere_rule()
    rng = np.random.default_rng(3)
    for _ in range(4):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        a = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 else [0.0, 1.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(n, a)
        dd = d[:, :1] * a + d[:, 1:2] * b + d[:, 2:] * n
        t = rng.normal(size=3)
        t -= t.dot(n) * n
        t /= np.linalg.norm(t)
        ki = 0.6 * t - 0.8 * n
        for pat, aR, aI, lam in ((0, 1, 1, 1.0), (1, 4, 1, 1.0), (2, 3, 5, 0.4)):
            f = orc.scat_pattern(pat, ki, n, dd, aR, aI, lam)
            assert abs((f * W).sum() - 1.0) < 1e-9


def test_directive_alpha1_closed_form(orc):
    # F_1 = (I_0 + I_1) / 2 = (2 pi + pi cos theta_i) / 2, worked out by hand from
    # Eq. directive_model; the pattern peaks at 1 / F_1 in the specular direction
    n = np.array([0.0, 0.0, 1.0])
    for th_i in (0.0, 0.5, 1.3):
        c = math.cos(th_i)
        assert abs(orc.f_alpha(1, c) - (math.pi + 0.5 * math.pi * c)) < 1e-14
        ki = np.array([math.sin(th_i), 0.0, -c])
        kr = np.array([math.sin(th_i), 0.0, c])
        assert abs(orc.scat_pattern(1, ki, n, kr)[0] * (math.pi + 0.5 * math.pi * c) - 1.0) < 1e-14
    # alpha = 2: F_2 = (I_0 + 2 I_1 + I_2) / 4 = (2 pi + 2 pi c + 2 pi / 3) / 4
    for c in (1.0, 0.4):
        assert abs(orc.f_alpha(2, c) - (2 * math.pi + 2 * math.pi * c + 2 * math.pi / 3) / 4) < 1e-14
    # alpha = 3 adds I_3 = (pi / 2) c (1 + sin^2 / 2)
    c = 0.7
    s2 = 1 - c * c
    F3 = (2 * math.pi + 3 * math.pi * c + 3 * 2 * math.pi / 3 + math.pi / 2 * c * (1 + s2 / 2)) / 8
    assert abs(orc.f_alpha(3, c) - F3) < 1e-13


def test_backscattering_limits(orc):
    d, _ = _hemisphere_rule(8, 16)
    n = np.array([0.0, 0.0, 1.0])
    ki = np.array([0.6, 0.0, -0.8])
    # Lambda = 1 reduces to the directive model
    assert np.allclose(orc.scat_pattern(2, ki, n, d, 4, 9, 1.0), orc.scat_pattern(1, ki, n, d, 4), rtol=1e-14)
    # Lambda = 0 is a lobe around -k_i, peaking there
    f = orc.scat_pattern(2, ki, n, np.vstack([d, -ki]), 3, 6, 0.0)
    assert f[-1] >= f[:-1].max()
    # Lambertian does not depend on the incidence direction
    assert np.array_equal(orc.scat_pattern(0, ki, n, d), orc.scat_pattern(0, np.array([0, 0, -1.0]), n, d))


# ---------------------------------------------------------------------------
# hemisphere sampler
# ---------------------------------------------------------------------------
def test_diffuse_direction_is_uniform_on_hemisphere(orc):
    m = 64
    g = (np.arange(m) + 0.5) / m
    U = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    rng = np.random.default_rng(1)
    normals = [np.array(v, float) for v in ([0, 0, 1], [0, 0, -1], [1, 0, 0], [0, -1, 0],
                                           [0, 0.8, -0.6], [0.3, 0.4, -0.5])]
    normals += [rng.normal(size=3) for _ in range(3)]
    for n in normals:
        n = n / np.linalg.norm(n)
        d = orc.diffuse_dir(n, U)
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
        # cos theta_s = 1 - u1 exactly (uniform in cos theta <=> uniform in solid angle)
        assert np.allclose(d @ n, 1.0 - U[:, 0], atol=1e-14)
        # midpoint rule over the unit square = the hemisphere average:
        # E[k] = n / 2, E[k k^T] = I / 3 (every second moment of a uniform
        # hemisphere equals that of the sphere)
        assert np.allclose(d.mean(0), n / 2, atol=1e-3)
        assert np.allclose(d.T @ d / len(d), np.eye(3) / 3, atol=1e-3)
        # the azimuth advances by 2 pi (u2' - u2)
        a = orc.diffuse_dir(n, [[0.5, 0.1], [0.5, 0.35]])
        pa = a - np.outer(a @ n, n)
        cosang = pa[0] @ pa[1] / (np.linalg.norm(pa[0]) * np.linalg.norm(pa[1]))
        assert abs(cosang - math.cos(2 * math.pi * 0.25)) < 1e-12


# ---------------------------------------------------------------------------
# scattered field (Eq. scattered_field)
# ---------------------------------------------------------------------------
def _r_half_space(eta, c):
    s = np.sqrt(eta - (1 - c * c) + 0j)
    return (c - s) / (c + s), (eta * c - s) / (eta * c + s)


def test_scattered_field_power_and_transversality(orc):
    f, eps, sig = 28e9, 5.0, 0.05
    eta = eps - 1j * sig / (EPS0 * 2 * math.pi * f)
    n = np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(7)
    for trial in range(20):
        th = rng.uniform(0.05, 1.45)
        k = np.array([math.sin(th), 0.0, -math.cos(th)])
        e_perp = np.array([0.0, 1.0, 0.0])               # k x n / |k x n| for this geometry
        e_par = np.cross(e_perp, k)
        a, b = rng.normal(size=2) + 1j * rng.normal(size=2)
        E = a * e_perp + b * e_par
        Sd, Kx = rng.uniform(0.1, 1.0), rng.uniform(0, 1)
        pat, aR, aI, lam = trial % 3, 1 + trial % 5, 2, 0.5
        u = rng.uniform(size=4)
        ks, Es = orc.diffuse_interact(k, n, E, eps, sig, f, 0.0, Sd, Kx, pat, aR, aI, lam, u)
        fs = orc.scat_pattern(pat, k, n, ks, aR, aI, lam)[0]
        rp, rl = _r_half_space(eta, math.cos(th))
        want = 2 * math.pi * fs * Sd ** 2 * (abs(rp * a) ** 2 + abs(rl * b) ** 2)
        assert abs(np.vdot(Es, Es).real - want) <= 1e-12 * want
        assert abs(Es @ ks) <= 1e-13 * np.linalg.norm(Es)


def _sph(k):
    t, p = math.acos(k[2]), math.atan2(k[1], k[0])
    return (np.array([math.cos(t) * math.cos(p), math.cos(t) * math.sin(p), -math.sin(t)]),
            np.array([-math.sin(p), math.cos(p), 0.0]))


def test_cross_polarisation_split(orc):
    # the matrix [[sqrt(1-K), -sqrt(K)], [sqrt(K), sqrt(1-K)]] acting on (E_theta, E_phi)
    k = np.array([0.6, 0.0, -0.8])
    n = np.array([0.0, 0.0, 1.0])
    th_i, ph_i = _sph(k)
    u = (0.4, 0.3, 0.0, 0.0)                              # chi_1 = chi_2 = 0
    for E, K, frac_theta in ((th_i, 0.0, 1.0), (th_i, 1.0, 0.0), (th_i, 0.3, 0.7), (ph_i, 0.3, 0.3),
                             ((th_i + ph_i) / math.sqrt(2), 0.5, 0.0)):
        ks, Es = orc.diffuse_interact(k, n, E.astype(complex), 4.0, 0.0, 3.5e9, 0.0, 1.0, K, 0, 1, 1, 1.0, u)
        th_s, _ = _sph(ks)
        p = np.vdot(Es, Es).real
        assert abs(abs(th_s @ Es) ** 2 / p - frac_theta) < 1e-12, (K, frac_theta)
    # the random phases multiply the two rows: with K = 0 the theta row gets e^{j chi_1}
    E = th_i.astype(complex)
    _, e0 = orc.diffuse_interact(k, n, E, 4.0, 0.0, 3.5e9, 0.0, 1.0, 0.0, 0, 1, 1, 1.0, (0.4, 0.3, 0.0, 0.0))
    _, e1 = orc.diffuse_interact(k, n, E, 4.0, 0.0, 3.5e9, 0.0, 1.0, 0.0, 0, 1, 1, 1.0, (0.4, 0.3, 0.25, 0.6))
    assert np.allclose(e1, 1j * e0, atol=1e-14)


# ---------------------------------------------------------------------------
# energy bookkeeping and the map of a Lambertian ground
# ---------------------------------------------------------------------------
def test_lossless_closed_box_conserves_power_in_expectation(orc):
    # lossless slab walls: R + S + T carry all incident power, so the mean over
    # seeds of (power alive at segment l + power escaped before) is N
    sc = S.closed_box(10.0, mat=(3.0, 0.0, 0.2)).with_scattering(0.6, 0.2, [2], 3, 2, 0.7)
    N, L = 400, 5
    p = S.TraceParams(28e9, L, cell_size=1.0, nx=8, ny=8, map_origin=(0, 0, -2.0), diffuse=True)
    tot = []
    n_diff = 0
    for seed in range(48):
        r = orc.radio_map(sc, S.Tx(pos=(1.0, 2.0, 3.0), num_rays=N, seed=seed), p, stats=True, want_record=True)
        pw, esc = r["power"], r["escaped"]
        tot.append([pw[l] + esc[:l].sum() for l in range(L + 1)])
        n_diff += int((r["record"][:, :, 3] & 3 == 2).sum())
    tot = np.array(tot)
    m, se = tot.mean(0), tot.std(0, ddof=1) / math.sqrt(len(tot))
    assert abs(m[0] - N) < 1e-9 * N
    assert np.all(np.abs(m[1:] - N) <= 4.5 * se[1:] + 1e-9 * N), (m, se)
    assert n_diff > 1000


def test_lambertian_ground_map_matches_quadrature(orc):
    """Diffuse-only map (S = 1, no LoS) over a Lambertian ground against the
    model's integral C(t) = (lambda0/4pi)^2 S^2 int Gamma^2 f_s cos(theta_i) /
    (r0^2 d1^2) dA, with f_s = cos(theta_s) / pi and, for a V-pol isotropic TX
    over horizontal ground (TM incidence), Gamma^2 = |r_par(theta_i)|^2."""
    f, H, h = 3.5e9, 20.0, 1.5
    eps, sig = 5.24, 0.0462
    lam0 = C0 / f
    eta = eps - 1j * sig / (EPS0 * 2 * math.pi * f)
    sc = S.ground_plane().with_scattering(1.0)
    N = 3_000_000
    cell, nx = 4.0, 16
    p = S.TraceParams(f, 1, los=False, refract=False, cell_size=cell, nx=nx, ny=nx, diffuse=True)
    got = orc.radio_map(sc, S.Tx(pos=(0.0, 0.0, H), num_rays=N, seed=3), p)["map"]

    # inner integral in polar coordinates about t: rho = h tan(beta) turns
    # h / d1^3 dA into sin(beta) d(beta) d(psi)
    gb, wb = np.polynomial.legendre.leggauss(160)
    beta = (gb + 1) * np.pi / 4
    wbeta = wb * np.pi / 4 * np.sin(beta)
    npsi = 96
    psi = np.arange(npsi) * 2 * np.pi / npsi

    def C_at(tx_, ty_):
        rho = h * np.tan(beta)[:, None]
        qx = tx_ + rho * np.cos(psi)[None, :]
        qy = ty_ + rho * np.sin(psi)[None, :]
        r0 = np.sqrt(qx ** 2 + qy ** 2 + H * H)
        c = H / r0
        s = np.sqrt(eta - (1 - c * c) + 0j)
        g2 = np.abs((eta * c - s) / (eta * c + s)) ** 2
        inner = (g2 * c / r0 ** 2 * wbeta[:, None]).sum() * 2 * np.pi / npsi
        return (lam0 / (4 * math.pi)) ** 2 / math.pi * inner

    gc, wc = np.polynomial.legendre.leggauss(3)
    x0 = -0.5 * nx * cell
    checked = 0
    for iy in range(nx):
        for ix in range(nx):
            xs = x0 + (ix + (gc + 1) / 2) * cell
            ys = x0 + (iy + (gc + 1) / 2) * cell
            want = sum(wc[a] * wc[b] / 4 * C_at(xs[a], ys[b]) for a in range(3) for b in range(3))
            # rays per cell: N / (4 pi) per sr over ~ H^2 / cos^3 m^2 of ground per sr
            rho = math.hypot(xs.mean(), ys.mean())
            n_exp = N / (4 * math.pi) * cell * cell * (H / math.hypot(rho, H)) ** 3 / H ** 2
            if n_exp < 2000:
                continue
            assert abs(got[iy, ix] - want) <= 5.0 / math.sqrt(n_exp) * want, (ix, iy, got[iy, ix], want)
            checked += 1
    assert checked >= 100


# ---------------------------------------------------------------------------
# modes
# ---------------------------------------------------------------------------
def _diffuse_manhattan(stride=997):
    sc, txs, p = S.workload(2)
    sc = sc.with_scattering(np.linspace(0.3, 0.7, sc.nm), 0.2, np.arange(sc.nm) % 3, 3, 2, 0.6)
    tx = txs[0]
    tx.ray_stride = stride
    p.nx = p.ny = 128
    p.cell_size = 4.0
    p.diffuse = True
    return sc, tx, p


def test_scattering_zero_is_specular_bit_for_bit(orc):
    sc, tx, p = _diffuse_manhattan()
    a = orc.radio_map(sc.with_scattering(0.0), tx, p)["map"]
    p0 = copy.copy(p)
    p0.diffuse = False
    b = orc.radio_map(sc, tx, p0)["map"]
    c = orc.radio_map(S.workload(2)[0], tx, p0)["map"]
    assert np.array_equal(a, c) and np.array_equal(b, c)


def test_diffuse_replay_frozen_and_planted_decision(orc):
    sc, tx, p = _diffuse_manhattan()
    a = orc.radio_map(sc, tx, p, want_record=True)
    rec = a["record"]
    dec = rec[:, :, 3]
    assert ((dec >= 0) & (dec & 3 == 2)).sum() > 100
    b = orc.radio_map(sc, tx, p, mode="replay", record=rec)
    assert b["report"]["failures"] == 0 and np.array_equal(a["map"], b["map"])
    c = orc.radio_map(sc, tx, p, mode="frozen", record=rec)
    assert np.array_equal(a["map"], c["map"])
    # a diffuse choice planted where the coin was far from the S interval fails
    spec = np.argwhere(dec == 0)
    u = np.array([orc.rng_u(tx.seed, tx.ray_begin + i * tx.ray_stride, l) for i, l in spec])
    i, l = spec[np.argmin(u)]
    assert u.min() < 0.01
    bad = rec.copy()
    bad[i, l, 3] = 2
    rep = orc.radio_map(sc, tx, p, mode="replay", record=bad)["report"]
    assert rep["failures"] >= 1 and rep["fail_kind"] == 3


def test_branch_all_refuses_diffuse(orc):
    sc, tx, p = _diffuse_manhattan()
    with pytest.raises(ValueError):
        orc.branch_all(sc, tx, p)


def test_invalid_scattering_parameters_are_rejected(orc):
    sc, tx, p = _diffuse_manhattan()
    for bad in (dict(S=1.5), dict(S=0.5, K_x=-0.1), dict(S=0.5, pattern=3), dict(S=0.5, pattern=1, alpha_r=0),
                dict(S=0.5, pattern=2, lam=2.0)):
        with pytest.raises(ValueError):
            orc.radio_map(sc.with_scattering(**bad), tx, p)


@pytest.mark.parametrize("deposit", [1, 0])
def test_grad_dual_matches_frozen_fd_with_diffuse(orc, deposit):
    sc, txs, p = S.workload(4)
    sc = sc.with_scattering(np.linspace(0.2, 0.8, sc.nm), 0.3, np.arange(sc.nm) % 3, 2, 3, 0.5)
    tx = txs[0]
    tx.ray_stride, tx.ray_count = 331, 3000
    p.deposit = deposit
    p.nx = p.ny = 96
    p.diffuse = True
    base = orc.radio_map(sc, tx, p, want_record=True)
    rec = base["record"]
    assert ((rec[:, :, 3] >= 0) & (rec[:, :, 3] & 3 == 2)).sum() > 50
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
