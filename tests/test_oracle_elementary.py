"""Pins of the oracle's elementary functions against closed forms, identities,
library routines and published vectors (CPU only)."""
import cmath
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

EPS0 = 8.8541878128e-12
C0 = 299792458.0
HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# complex square root (principal branch) vs the C library's csqrt
# ---------------------------------------------------------------------------
def test_csqrt_matches_library(orc):
    rng = np.random.default_rng(1)
    zs = list(rng.normal(size=200) * 10 + 1j * rng.normal(size=200) * 10)
    zs += [complex(-4.0, 0.0), complex(-4.0, -0.0), complex(0.0, -3.0), complex(5.24, -0.237),
           complex(1e-300, -1e-300), complex(1e150, -1e149), complex(-1e-3, 1e-20), complex(3.0, 0.0)]
    for z in zs:
        a, b = orc.csqrt(z), cmath.sqrt(z)
        assert abs(a - b) <= 1e-15 * abs(b) + 1e-300, (z, a, b)


# ---------------------------------------------------------------------------
# Fresnel coefficients for incidence from vacuum (Eq. fresnel_vac)
# ---------------------------------------------------------------------------
MATS = [(5.24, 0.0462, 3.5e9), (4.0, 0.0, 28e9), (3.0, 0.5, 28e9), (6.5, 0.01, 28e9), (1.5, 1e-3, 2.4e9)]


@pytest.mark.parametrize("er,sig,f", MATS)
def test_fresnel_normal_incidence(orc, er, sig, f):
    eta = er - 1j * sig / (EPS0 * 2 * math.pi * f)
    rp, rl, _, _ = orc.fresnel(er, sig, f, 1.0)
    ref = (cmath.sqrt(eta) - 1) / (cmath.sqrt(eta) + 1)
    assert abs(rl - ref) < 1e-14 and abs(rp + ref) < 1e-14


@pytest.mark.parametrize("er,sig,f", MATS)
def test_fresnel_grazing_limit(orc, er, sig, f):
    rp, rl, _, _ = orc.fresnel(er, sig, f, 1e-9)
    assert abs(rp + 1) < 1e-8 and abs(rl + 1) < 1e-8


@pytest.mark.parametrize("er", [2.0, 4.0, 7.5])
def test_fresnel_brewster_zero(orc, er):
    # lossless: r_par vanishes at tan(theta_B) = sqrt(eta)
    c = 1.0 / math.sqrt(1.0 + er)
    _, rl, _, _ = orc.fresnel(er, 0.0, 1e9, c)
    assert abs(rl) < 1e-14


@pytest.mark.parametrize("er", [2.0, 4.0, 7.5])
def test_fresnel_textbook_snell_and_energy(orc, er):
    # Textbook form with the refraction angle from Snell's law (real index n),
    # and power conservation at the interface |r|^2 + (n cos2 / cos1) |t|^2 = 1.
    n = math.sqrt(er)
    for th1 in np.linspace(0.0, 1.5, 13):
        c1 = math.cos(th1)
        th2 = math.asin(math.sin(th1) / n)
        c2 = math.cos(th2)
        rp, rl, _, _ = orc.fresnel(er, 0.0, 1e9, c1)
        tp, tl = orc.fresnel_vac_t(er, 0.0, 1e9, c1)
        assert abs(rp - (c1 - n * c2) / (c1 + n * c2)) < 1e-14
        assert abs(rl - (n * c1 - c2) / (n * c1 + c2)) < 1e-14
        assert abs(tp - 2 * c1 / (c1 + n * c2)) < 1e-14
        assert abs(tl - 2 * c1 / (c2 + n * c1)) < 1e-14
        assert abs(abs(rp) ** 2 + n * c2 / c1 * abs(tp) ** 2 - 1) < 1e-13
        assert abs(abs(rl) ** 2 + n * c2 / c1 * abs(tl) ** 2 - 1) < 1e-13


# ---------------------------------------------------------------------------
# Single-layer slab (Eqs. fresnel_slab, q_fresnel_slab)
# ---------------------------------------------------------------------------
def _char_matrix(eta, c1, k0d, pol):
    """Born & Wolf characteristic-matrix reflection / transmission of a layer in vacuum.

    TE: admittances Y = n cos2 (layer), Y0 = cos1 (vacuum); TM: tilted
    admittances n / cos2 and 1 / cos1, coefficients of the tangential field.
    """
    s1 = math.sqrt(max(0.0, 1 - c1 * c1))
    n = np.sqrt(complex(eta))
    c2 = np.sqrt(1 - s1 * s1 / eta)
    d = k0d * n * c2
    Y = n * c2 if pol == "te" else n / c2
    Y0 = c1 if pol == "te" else 1.0 / c1
    m11, m12, m21, m22 = np.cos(d), 1j * np.sin(d) / Y, 1j * Y * np.sin(d), np.cos(d)
    den = Y0 * m11 + Y0 * Y0 * m12 + m21 + Y0 * m22
    return (Y0 * m11 + Y0 * Y0 * m12 - m21 - Y0 * m22) / den, 2 * Y0 / den


@pytest.mark.parametrize("er,sig", [(4.0, 0.0), (5.0, 0.01), (3.0, 0.5), (6.9, 0.9)])
@pytest.mark.parametrize("c1", [1.0, 0.8, 0.3, 0.05])
def test_slab_matches_characteristic_matrix(orc, er, sig, c1):
    f, d = 28e9, 0.2
    eta = er - 1j * sig / (EPS0 * 2 * math.pi * f)
    k0d = 2 * math.pi * f / C0 * d
    rp, rl, tp, tl = orc.fresnel(er, sig, f, c1, d)
    r_te, t_te = _char_matrix(eta, c1, k0d, "te")
    r_tm, t_tm = _char_matrix(eta, c1, k0d, "tm")
    assert abs(rp - r_te) < 1e-12 and abs(tp - t_te) < 1e-12
    # TM: the characteristic matrix reports the tangential-field ratio, whose
    # reflected part has the opposite sign convention to the TM amplitude.
    assert abs(rl + r_tm) < 1e-12 and abs(tl - t_tm) < 1e-12


@pytest.mark.parametrize("er", [1.7, 3.0, 5.24, 7.0])
def test_slab_lossless_energy(orc, er):
    for d in (0.01, 0.2, 1.37):
        for c1 in np.linspace(0.02, 1.0, 17):
            rp, rl, tp, tl = orc.fresnel(er, 0.0, 28e9, c1, d)
            assert abs(abs(rp) ** 2 + abs(tp) ** 2 - 1) < 1e-13
            assert abs(abs(rl) ** 2 + abs(tl) ** 2 - 1) < 1e-13


def test_slab_thin_and_thick_limits(orc):
    for c1 in (1.0, 0.6, 0.1):
        rp, rl, tp, tl = orc.fresnel(5.0, 0.1, 28e9, c1, 1e-14)
        assert abs(rp) < 1e-9 and abs(rl) < 1e-9 and abs(tp - 1) < 1e-9 and abs(tl - 1) < 1e-9
        hp, hl, _, _ = orc.fresnel(5.0, 1.0, 28e9, c1, 0.0)
        rp, rl, tp, tl = orc.fresnel(5.0, 1.0, 28e9, c1, 5.0)
        assert abs(rp - hp) < 1e-12 and abs(rl - hl) < 1e-12 and abs(tp) < 1e-12 and abs(tl) < 1e-12


# ---------------------------------------------------------------------------
# counter-based RNG
# ---------------------------------------------------------------------------
def test_splitmix64_published_vectors(orc):
    lines = [l for l in open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) if not l.startswith("#")]
    want = [int(l, 16) for l in lines if l.strip()]
    G = 0x9E3779B97F4A7C15
    got = [orc.splitmix64((k * G) & ((1 << 64) - 1)) for k in range(3)]
    assert got == want


def test_rng_uniform_24bit(orc):
    us = np.array([orc.rng_u(7, n, l) for n in range(20000) for l in range(4)])
    assert us.min() >= 0.0 and us.max() < 1.0
    assert np.all(us * 2 ** 24 == np.floor(us * 2 ** 24))
    # mean and a 16-bin chi-square
    assert abs(us.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(us))
    h, _ = np.histogram(us, bins=16, range=(0, 1))
    e = len(us) / 16
    chi2 = ((h - e) ** 2 / e).sum()
    assert chi2 < 45  # 15 dof, p ~ 1e-4
    # distinct seeds decorrelate
    a = np.array([orc.rng_u(1, n, 0) for n in range(5000)])
    b = np.array([orc.rng_u(2, n, 0) for n in range(5000)])
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.06


# ---------------------------------------------------------------------------
# Fibonacci lattice (Sec. 3.1.1)
# ---------------------------------------------------------------------------
def test_fibonacci_definition_high_precision(orc):
    getcontext().prec = 60
    phi_g = (1 + Decimal(5).sqrt()) / 2
    for N in (2, 3, 1000, 10 ** 7, 10 ** 9):
        ns = sorted({0, 1, N // 3, N // 2, N - 2, N - 1} | {int(x) for x in np.linspace(0, N - 1, 25)})
        ns = [n for n in ns if 0 <= n < N]
        for n in ns:
            k = orc.fibonacci(N, n, 1, 1)[0]
            z = 1 - 2 * n / (N - 1)
            assert abs(k[2] - z) <= 2e-16
            assert abs(np.linalg.norm(k) - 1) < 1e-15
            q = Decimal(n) / phi_g
            frac = float(q - int(q))
            st = math.sqrt(max(0.0, (1 - z) * (1 + z)))
            if st > 1e-6:
                ph = math.atan2(k[1], k[0]) % (2 * math.pi)
                d = abs(ph - 2 * math.pi * frac)
                # W = round(2^64 (phi_g - 1)) is exact to 2^-65, so n W mod 2^64
                # is within n 2^-65 of a turn of the exact fractional part
                tol = 2 * math.pi * (n + 1) * 2.0 ** -65 + 1e-12
                assert min(d, 2 * math.pi - d) < tol, (N, n)


def test_fibonacci_single_and_uniform(orc):
    k = orc.fibonacci(1)
    assert np.allclose(k, [[-1.0, 0.0, 0.0]], atol=1e-15)
    N = 200000
    d = orc.fibonacci(N)
    assert np.abs(d.mean(0)).max() < 1e-4
    # equal-area: points in a cap of half-angle a around the x axis ~ N (1 - cos a) / 2
    for a in (0.2, 0.7, 1.5):
        frac = np.mean(d[:, 0] > math.cos(a))
        assert abs(frac - (1 - math.cos(a)) / 2) < 5 / math.sqrt(N)


# ---------------------------------------------------------------------------
# orientation and antenna pattern (App. A.1, Eq. C)
# ---------------------------------------------------------------------------
def test_rotation_matches_scipy(orc):
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(3)
    for _ in range(20):
        a, b, g = rng.uniform(-math.pi, math.pi, 3)
        R = orc.rotation(a, b, g)
        ref = Rotation.from_euler("ZYX", [a, b, g]).as_matrix()
        assert np.abs(R - ref).max() < 1e-14


def test_tx_field_isotropic_vertical_is_theta_hat(orc):
    d = orc.fibonacci(5001)[1:-1]
    E = orc.tx_field(d, pattern=0, pol=0)
    th = np.arccos(d[:, 2])
    ph = np.arctan2(d[:, 1], d[:, 0])
    ref = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], 1)
    assert np.abs(E - ref).max() < 1e-12
    H = orc.tx_field(d, pattern=0, pol=1)
    assert np.abs(H - np.stack([-np.sin(ph), np.cos(ph), 0 * ph], 1)).max() < 1e-12


def test_tx_pattern_normalisation_and_orientation(orc):
    # G = |C|^2 integrates to 4 pi over the sphere (product Gauss-Legendre rule);
    # the field is transverse and a rotated dipole has G = 1.5 sin^2 of the
    # angle to its rotated axis.
    x, w = np.polynomial.legendre.leggauss(64)
    phs = np.linspace(0, 2 * math.pi, 128, endpoint=False)
    Z, P = np.meshgrid(x, phs, indexing="ij")
    st = np.sqrt(1 - Z ** 2)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), Z], -1).reshape(-1, 3)
    W = (w[:, None] * np.full(len(phs), 2 * math.pi / len(phs))[None, :]).reshape(-1)
    for pattern in (0, 1):
        for (a, b, g) in ((0, 0, 0), (0.3, -1.1, 2.0), (2.5, 0.4, -0.7)):
            for pol in (0, 1):
                E = orc.tx_field(dirs, a, b, g, pattern, pol)
                G = (E ** 2).sum(1)
                assert abs((G * W).sum() - 4 * math.pi) < 1e-9
                assert np.abs((E * dirs).sum(1)).max() < 1e-12
                if pattern == 1:
                    axis = orc.rotation(a, b, g)[:, 2]
                    c = dirs @ axis
                    assert np.abs(G - 1.5 * (1 - c ** 2)).max() < 1e-12


# ---------------------------------------------------------------------------
# field update at one interface (App. A.7 basis vectors)
# ---------------------------------------------------------------------------
def test_interact_normal_incidence_any_basis(orc):
    k = np.array([0.0, 0.0, -1.0])
    n = np.array([0.0, 0.0, 1.0])
    rp, rl, _, _ = orc.fresnel(5.0, 0.2, 28e9, 1.0)
    for E in ([1, 0, 0], [0, 1, 0], [0.6, 0.8j, 0], [1 + 2j, -0.5, 0]):
        ko, Eo = orc.interact(k, n, E, 5.0, 0.2, 28e9, 0.0, 0)
        assert np.allclose(ko, [0, 0, 1], atol=1e-15)
        assert np.abs(Eo - rp * np.asarray(E)).max() < 1e-14
        assert abs(rl + rp) < 1e-14


def test_interact_te_tm_and_power(orc):
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        k = rng.normal(size=3)
        k /= np.linalg.norm(k)
        if abs(k @ n) < 0.05:
            continue
        nn = n if k @ n < 0 else -n
        c1 = -k @ nn
        e_perp = np.cross(k, nn)
        e_perp /= np.linalg.norm(e_perp)
        e_par = np.cross(e_perp, k)
        a, b = rng.normal(size=2) + 1j * rng.normal(size=2)
        E = a * e_perp + b * e_par
        for thick, dec in ((0.0, 0), (0.2, 0), (0.2, 1)):
            rp, rl, tp, tl = orc.fresnel(4.5, 0.05, 28e9, c1, thick)
            ko, Eo = orc.interact(k, n, E, 4.5, 0.05, 28e9, thick, dec)
            ko2, Eo2 = orc.interact(k, -n, E, 4.5, 0.05, 28e9, thick, dec)
            assert np.abs(Eo - Eo2).max() < 1e-13 and np.abs(ko - ko2).max() < 1e-15
            kref = k - 2 * (k @ nn) * nn if dec == 0 else k
            assert np.abs(ko - kref).max() < 1e-14
            assert abs(Eo @ ko) < 1e-13  # transverse
            cp, cl = (rp, rl) if dec == 0 else (tp, tl)
            assert abs(Eo @ e_perp - cp * a) < 1e-13  # TE component keeps its basis vector
            assert abs(np.vdot(Eo, Eo).real - (abs(cp * a) ** 2 + abs(cl * b) ** 2)) < 1e-12
