"""Pins of the oracle's first-order diffraction radio map (Sec. 4, "Computation
of Radio Map due to Diffraction", estimator Eq. radio-map-solver-ci-D-est;
UTD of App. A.8, Eq. diffracted-field; weighting factor of the appendix on
diffraction radio maps): the transition function against the standard
Fresnel integrals, the wedges of a box, the weighting factor against finite
differences, the UTD field's jumps at the incident and reflection shadow
boundaries (which must cancel the geometrical-optics field's), and the
estimator against a direct integration of the map's definition over cells."""
import math

import numpy as np
import pytest
import scipy.special as sps

from synth import scenes as S

C0 = 299792458.0
EPS0 = 8.8541878128e-12


# ---------------------------------------------------------------------------
# transition function
# ---------------------------------------------------------------------------
def test_transition_function_matches_fresnel_integrals(orc):
    # F(x) = sqrt(pi x / 2) e^{jx} [1 + j - 2 (S(sqrt(2x/pi)) + j C(sqrt(2x/pi)))], S, C the
    # standard Fresnel integrals (scipy)
    for x in np.concatenate([np.logspace(-6, 6, 61), [0.5, 1.0, 2.0, 7.3]]):
        Sx, Cx = sps.fresnel(math.sqrt(2 * x / math.pi))
        ref = math.sqrt(math.pi * x / 2) * np.exp(1j * x) * (1 + 1j - 2 * (Sx + 1j * Cx))
        got = orc.utd_F(x)
        assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (x, got, ref)
    assert orc.utd_F(0.0) == 0
    # limits: F -> 1 for large x; F ~ sqrt(pi x) e^{j pi/4} for small x
    assert abs(orc.utd_F(1e8) - 1) < 1e-7
    x = 1e-10
    assert abs(orc.utd_F(x) / (math.sqrt(math.pi * x) * np.exp(1j * math.pi / 4)) - 1) < 1e-4


# ---------------------------------------------------------------------------
# wedges
# ---------------------------------------------------------------------------
def test_wedges_of_a_box(orc):
    sc = S.single_box(0.0, 20.0, 0.0, 30.0, 25.0)
    W = orc.wedges(sc)
    assert len(W) == 12
    assert np.allclose(W[:, 13], 1.5)                     # right-angle corners: exterior angle 3 pi / 2
    assert sorted(np.round(W[:, 12]).astype(int)) == sorted([20] * 4 + [30] * 4 + [25] * 4)
    for w in W:
        e, n0, nn = w[3:6], w[6:9], w[9:12]
        assert np.allclose(np.cross(n0, nn), e)           # e = n0 x nn / |n0 x nn|
        assert abs(np.linalg.norm(e) - 1) < 1e-12 and abs(n0 @ nn) < 1e-12
        assert w[14] < w[15]                              # 0-face = lower triangle index
    # the edge lies on both faces: its end points satisfy both plane equations
    v, t = sc.verts.astype(np.float64), sc.tris
    for w in W:
        for tri, nf in ((int(w[14]), w[6:9]), (int(w[15]), w[9:12])):
            a = v[t[tri, 0]]
            for x in (0.0, w[12]):
                assert abs((w[0:3] + x * w[3:6] - a) @ nf) < 1e-9
    # a flat quad (two coplanar triangles) has no wedge
    assert len(orc.wedges(S.ground_plane())) == 0
    # adjacent boxes: 100 boxes of the Manhattan scene, 12 wedges each, ground excluded
    assert len(orc.wedges(S.workload(2)[0])) == 1200


# ---------------------------------------------------------------------------
# weighting factor |dt/dx x dt/dphi|
# ---------------------------------------------------------------------------
def test_weighting_factor_matches_finite_differences(orc):
    sc = S.single_box(0.0, 20.0, 0.0, 30.0, 25.0)
    W = orc.wedges(sc)
    rng = np.random.default_rng(2)
    checked = 0
    for s in ([-30.0, -20.0, 15.0], [45.0, 50.0, 40.0], [10.0, -40.0, 5.0]):
        for w in W:
            for _ in range(4):
                x, phi = rng.uniform(0.05, 0.95) * w[12], rng.uniform(0.05, 0.95) * w[13] * math.pi
                r = orc.diffraction_point(w, s, x, phi, 1.5)
                if r is None:
                    continue
                t, J = r
                h = 1e-5
                def T(xx, pp):
                    q = orc.diffraction_point(w, s, xx, pp, 1.5)
                    return None if q is None else q[0]
                a, b, c, d = T(x + h, phi), T(x - h, phi), T(x, phi + h), T(x, phi - h)
                if a is None or b is None or c is None or d is None:
                    continue
                # central differences, Richardson-extrapolated
                a2, b2, c2, d2 = T(x + 2 * h, phi), T(x - 2 * h, phi), T(x, phi + 2 * h), T(x, phi - 2 * h)
                if a2 is None or b2 is None or c2 is None or d2 is None:
                    continue
                tx = (8 * (a - b) - (a2 - b2)) / (12 * h)
                tp = (8 * (c - d) - (c2 - d2)) / (12 * h)
                Jfd = np.linalg.norm(np.cross(tx, tp))
                assert abs(t[2] - 1.5) < 1e-9
                assert abs(J - Jfd) <= 1e-5 * Jfd, (J, Jfd)
                checked += 1
    assert checked > 40


# ---------------------------------------------------------------------------
# UTD field: shadow-boundary jumps (App. A.8)
# ---------------------------------------------------------------------------
def _oriented(w, s):
    o, e, n0, nn, L = w[0:3], w[3:6], w[6:9], w[9:12], w[12]
    if np.dot(s - o, n0) >= 0:
        return o, e, n0, nn
    return o + e * L, -e, nn, n0


def _keller_dir(e, t0, n0, beta_cos, phi):
    sb = math.sqrt(1 - beta_cos ** 2)
    return sb * (math.cos(phi) * t0 + math.sin(phi) * n0) + beta_cos * e


def _r_half_space(eta, c):
    s = np.sqrt(eta - (1 - c * c) + 0j)
    return (c - s) / (c + s), (eta * c - s) / (eta * c + s)


@pytest.mark.parametrize("src,pol", [((-30.0, -20.0, 15.0), 0), ((-25.0, 12.0, 40.0), 1), ((5.0, -35.0, 3.0), 0)])
def test_incident_shadow_boundary_jump_cancels_go_field(orc, src, pol):
    """Across phi = phi' + pi the diffracted field jumps by exactly the incident
    (geometrical-optics) field, so that GO + diffraction is continuous."""
    f = 3.5e9
    sc = S.single_box(0.0, 20.0, 0.0, 30.0, 25.0)
    s = np.array(src)
    n_checked = 0
    for w in orc.wedges(sc):
        o, e, n0, nn = _oriented(w, s)
        if np.dot(s - o, n0) < 0:
            continue
        t0 = np.cross(n0, e)
        v = o + 0.37 * w[12] * e
        sp = (v - s) / np.linalg.norm(v - s)
        st = (s - v) - ((s - v) @ e) * e
        phip = math.atan2(st @ n0, st @ t0) % (2 * math.pi)
        if phip + math.pi >= w[13] * math.pi - 1e-3:
            continue                                       # the ISB lies outside the exterior region
        E = orc.tx_field(sp, pol=pol)[0].astype(complex)
        sobs = 17.0
        dist = np.linalg.norm(v - s) + sobs
        out = []
        for sg in (+1, -1):
            sd = _keller_dir(e, t0, n0, sp @ e, phip + math.pi + sg * 1e-7)
            out.append(np.array(orc.utd_field(w, s, v, sd, sobs, E, mats=((5.0, 0.1), (5.0, 0.1)), freq_hz=f)))
        # beyond the ISB (phi > phi' + pi) the edge shadows the source: continuity of
        # GO + diffraction means E_d(shadow) - E_d(lit) = E_GO, resolved on the
        # diffracted basis (phi_hat, beta0_hat) = (-phi_hat', -beta0_hat') there
        jump = out[0] - out[1]
        go = np.linalg.norm(E) / dist
        ph = np.cross(sp, e)
        ph /= np.linalg.norm(ph)
        e_go = -np.array([ph @ E, np.cross(ph, sp) @ E]) / dist
        assert np.linalg.norm(jump - e_go) < 1e-4 * go, (jump, e_go)
        n_checked += 1
    assert n_checked >= 2


def test_reflection_shadow_boundary_jump(orc):
    """Across phi = pi - phi' (the specular direction off the 0-face) the
    diffracted field jumps by (minus) the 0-face's reflected field, built with
    the face's Fresnel coefficients (Eq. fresnel_vac) at cos theta = |n0 . s'|."""
    f = 28e9
    eps, sig = 5.0, 0.1
    eta = eps - 1j * sig / (EPS0 * 2 * math.pi * f)
    sc = S.single_box(0.0, 20.0, 0.0, 30.0, 25.0)
    n_checked = 0
    for src in ((-30.0, -20.0, 15.0), (40.0, 10.0, 30.0), (8.0, 45.0, 12.0)):
        s = np.array(src)
        for w in orc.wedges(sc):
            o, e, n0, nn = _oriented(w, s)
            if np.dot(s - o, n0) < 0:
                continue
            t0 = np.cross(n0, e)
            v = o + 0.61 * w[12] * e
            sp = (v - s) / np.linalg.norm(v - s)
            st = (s - v) - ((s - v) @ e) * e
            phip = math.atan2(st @ n0, st @ t0) % (2 * math.pi)
            rsb = math.pi - phip
            if not (1e-3 < rsb < w[13] * math.pi - 1e-3) or abs(rsb - (phip + math.pi)) < 1e-3:
                continue
            for pol in (0, 1):
                E = orc.tx_field(sp, pol=pol)[0].astype(complex)
                sobs = 23.0
                out = []
                for sg in (+1, -1):
                    sd = _keller_dir(e, t0, n0, sp @ e, rsb + sg * 1e-7)
                    out.append(np.array(orc.utd_field(w, s, v, sd, sobs, E, mats=((eps, sig), (eps, sig)), freq_hz=f)))
                # Near phi + phi' = pi, D_4 -> sgn(phi + phi' - pi) sqrt(L) / (2 sin b0) (cot ~ -2n/eps,
                # F(x) ~ sqrt(pi x) e^{j pi/4}), so Eq. diffracted-field jumps by -R_0 E_i / (s + s').
                # R_0 E_i is the reflected field r_perp a e_perp + r_par b (e_perp x s_r) of the 0-face
                # (Eqs. fresnel_in_vectors / fresnel_out_vectors) on the basis (phi_hat, beta0_hat)
                # of the specular direction s_r: the jump is minus that field.
                jump = out[0] - out[1]
                ep = np.cross(sp, n0)
                ep /= np.linalg.norm(ep)
                el = np.cross(ep, sp)
                sr = sp - 2 * (sp @ n0) * n0
                rp, rl = _r_half_space(eta, abs(n0 @ sp))
                er = rp * (ep @ E) * ep + rl * (el @ E) * np.cross(ep, sr)
                phd = -np.cross(sr, e)
                phd /= np.linalg.norm(phd)
                want = -np.array([phd @ er, np.cross(phd, sr) @ er]) / (np.linalg.norm(v - s) + sobs)
                assert np.linalg.norm(jump - want) < 1e-4 * np.linalg.norm(want), (jump, want)
                n_checked += 1
    assert n_checked >= 4


# ---------------------------------------------------------------------------
# estimator vs a direct integration of the definition (Eq. radio-map-solver-ci-D)
# ---------------------------------------------------------------------------
def _direct_gain(orc, W, s, T, f, mats):
    """Sum over wedges of e(p) at measurement points T [m, 3]: the diffraction
    point solves the Keller condition cos b0' = cos b0 on the edge (bisection;
    the difference is increasing along the edge), the diffracted direction must
    lie in the wedge's exterior, and e(p) = (lambda0/4pi)^2 |E_d|^2."""
    lam = C0 / f
    tot = np.zeros(len(T))
    for w in W:
        o, e, n0, nn = _oriented(w, s)
        if np.dot(s - o, n0) < 0:
            continue
        L, n = w[12], w[13]

        def fx(x):
            v = o[None] + x[:, None] * e[None]
            a = (v - s) @ e / np.linalg.norm(v - s, axis=1)
            b = np.einsum("ij,j->i", T - v, e) / np.linalg.norm(T - v, axis=1)
            return a - b

        lo, hi = np.zeros(len(T)), np.full(len(T), L)
        good = (fx(lo) <= 0) & (fx(hi) >= 0)
        for _ in range(60):
            m = 0.5 * (lo + hi)
            pos = fx(m) > 0
            hi, lo = np.where(pos, m, hi), np.where(pos, lo, m)
        V = o[None] + (0.5 * (lo + hi))[:, None] * e[None]
        t0 = np.cross(n0, e)
        for i in np.nonzero(good)[0]:
            sd = T[i] - V[i]
            d = np.linalg.norm(sd)
            sd /= d
            st = sd - (sd @ e) * e
            st /= np.linalg.norm(st)
            if math.atan2(st @ n0, st @ t0) % (2 * math.pi) > n * math.pi:
                continue
            sp = (V[i] - s) / np.linalg.norm(V[i] - s)
            E = orc.tx_field(sp)[0].astype(complex)
            ed = orc.utd_field(w, s, V[i], sd, d, E, mats=mats, freq_hz=f)
            tot[i] += (lam / (4 * math.pi)) ** 2 * (abs(ed[0]) ** 2 + abs(ed[1]) ** 2)
    return tot


def test_estimator_matches_direct_integration_of_the_definition(orc):
    """The (x, phi) estimator with its weighting factor against the map's
    definition, integrated directly over measurement points.  Cells that cut
    the building (where the integrand jumps at the walls) or carry under 1% of
    the largest value are left out; the quadrature's own error is estimated
    from two resolutions."""
    f = 3.5e9
    sc = S.single_box(0.0, 20.0, 0.0, 30.0, 25.0, mat=(5.0, 0.1, 0.2))
    p = S.TraceParams(f, 0, cell_size=4.0, nx=20, ny=20, map_origin=(10.0, 15.0, 1.5))
    s = np.array([-30.0, -20.0, 15.0])
    r = orc.diffraction_map(sc, S.Tx(pos=tuple(s), num_rays=1), p, 400_000, want_record=True)
    est, rec = r["map"], r["record"]
    cnt = np.zeros_like(est)
    ok = rec[:, 0] == 0
    np.add.at(cnt, (rec[ok, 2], rec[ok, 1]), 1)
    W = orc.wedges(sc)
    x0, y0 = p.map_corner()
    rels = []
    for k in np.argsort(-cnt.ravel()):
        iy, ix = divmod(int(k), p.nx)
        cx0, cy0 = x0 + ix * p.cell_size, y0 + iy * p.cell_size
        cuts = cx0 < 20.0 and cx0 + p.cell_size > 0.0 and cy0 < 30.0 and cy0 + p.cell_size > 0.0
        if cuts or est[iy, ix] < 0.01 * est.max():
            continue
        refs = []
        for m in (16, 32):
            g = (np.arange(m) + 0.5) / m
            X, Y = np.meshgrid(cx0 + g * p.cell_size, cy0 + g * p.cell_size)
            T = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 1.5)], 1)
            refs.append(_direct_gain(orc, W, s, T, f, ((5.0, 0.1), (5.0, 0.1))).mean())
        quad_err = abs(refs[1] - refs[0])
        assert abs(est[iy, ix] - refs[1]) <= 0.03 * refs[1] + 3 * quad_err, (ix, iy, est[iy, ix], refs)
        rels.append(abs(est[iy, ix] / refs[1] - 1))
        if len(rels) == 20:
            break
    assert len(rels) == 20
    assert np.median(rels) < 0.015, rels


# ---------------------------------------------------------------------------
# replay
# ---------------------------------------------------------------------------
def test_diffraction_replay_and_planted_visibility(orc):
    sc, txs, p = S.workload(2)
    p.nx = p.ny = 128
    p.cell_size = 4.0
    tx = txs[0]
    a = orc.diffraction_map(sc, tx, p, 64, want_record=True)
    rec = a["record"]
    assert a["visible"] > 1000 and (rec[:, 0] > 0).sum() > 1000   # blocked samples exist
    b = orc.diffraction_map(sc, tx, p, 64, mode="replay", record=rec)
    assert b["report"]["failures"] == 0 and np.array_equal(a["map"], b["map"])
    # a visible sample marked blocked, far from any graze, is rejected: a sample
    # from the middle of the lattice on a vertical edge (not grazing the ground)
    W = orc.wedges(sc)
    idx = np.arange(len(rec))
    cand = idx[(rec[:, 0] == 0) & (np.abs(W[idx // 64, 5]) == 1.0) & (idx % 64 >= 16) & (idx % 64 < 48)]
    assert len(cand)
    bad = rec.copy()
    bad[cand[len(cand) // 2], 0] = 2
    assert orc.diffraction_map(sc, tx, p, 64, mode="replay", record=bad)["report"]["failures"] == 1


def test_wedge_subsets_partition_the_map(orc):
    """The estimator is a sum over wedges: maps over a partition of the wedge
    list add up to the full map, and a subset's records are the full
    record's rows of those wedges, in the subset's order."""
    sc, txs, p = S.workload(2)
    p.nx = p.ny = 64
    p.cell_size = 8.0
    tx = txs[0]
    ns = 16
    full = orc.diffraction_map(sc, tx, p, ns, want_record=True)
    nw = len(orc.wedges(sc))
    rng = np.random.default_rng(11)
    perm = rng.permutation(nw)
    parts = [np.sort(perm[: nw // 3]), perm[nw // 3:]]          # the second part out of order
    total = np.zeros_like(full["map"])
    for idx in parts:
        r = orc.diffraction_map(sc, tx, p, ns, want_record=True, wedge_index=idx)
        rows = (idx[:, None] * ns + np.arange(ns)[None, :]).ravel()
        assert np.array_equal(r["record"], full["record"][rows])
        assert r["wedges"] == len(idx)
        total += r["map"]
    assert full["visible"] > 400
    assert np.allclose(total, full["map"], rtol=1e-12, atol=1e-12 * full["map"].max())
    with pytest.raises(ValueError):
        orc.diffraction_map(sc, tx, p, ns, wedge_index=[nw])


def test_mesh_wedge_subsets_partition_the_map(orc):
    """The same for the diffraction map on a mesh measurement surface."""
    from test_oracle_mesh import grid_surface
    sc, txs, p = S.workload(2)
    tx = txs[0]
    V, T = grid_surface(-64.0, -64.0, 8.0, 16, 16, lambda X, Y: 1.5 + 0.5 * np.sin(X / 9.0) * np.cos(Y / 7.0))
    ns = 8
    full = orc.diffraction_map_mesh(sc, tx, p, ns, V, T, want_record=True)
    nw = len(orc.wedges(sc))
    perm = np.random.default_rng(13).permutation(nw)
    parts = [np.sort(perm[: nw // 2]), perm[nw // 2:]]
    total = np.zeros_like(full["map"])
    for idx in parts:
        r = orc.diffraction_map_mesh(sc, tx, p, ns, V, T, want_record=True, wedge_index=idx)
        rows = (idx[:, None] * ns + np.arange(ns)[None, :]).ravel()
        assert np.array_equal(r["record"], full["record"][rows])
        total += r["map"]
    assert full["map"].max() > 0
    assert np.allclose(total, full["map"], rtol=1e-12, atol=1e-12 * full["map"].max())
