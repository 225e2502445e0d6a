"""Closed forms and statistics shared by the oracle pins and the GPU pins
(imported by tests only).  Nothing here calls the oracle or the CUDA path."""
import math

import numpy as np

from synth import scenes as S

C0 = 299792458.0
EPS0 = 8.8541878128e-12


def cell_avg(fn, x0, y0, cell, nx, ny, order=8):
    """Cell averages of fn(X, Y) by an order x order Gauss-Legendre rule."""
    g, w = np.polynomial.legendre.leggauss(order)
    W = np.outer(w, w) / 4.0
    out = np.zeros((ny, nx))
    for iy in range(ny):
        for ix in range(nx):
            xs = x0 + ix * cell + (g + 1) * cell / 2
            ys = y0 + iy * cell + (g + 1) * cell / 2
            X, Y = np.meshgrid(xs, ys)
            out[iy, ix] = (W * fn(X, Y)).sum()
    return out


def two_ray(tx_pos, params, num_rays, eps_r=5.24, sigma=0.0462):
    """Cell-averaged two-ray gain over a half-space ground for a V-polarised
    isotropic TX on the z axis, and the expected number of rays through each
    cell.  V-pol over horizontal ground is pure TM (theta-hat lies in the plane
    of incidence), so the reflected term carries |r_par|^2 only (Sec. A.5,
    vacuum-incident Fresnel coefficients); the two terms add non-coherently
    (Sec. 4.1).  Returns (gain [ny, nx], rays [ny, nx])."""
    f, ht, hr = params.freq_hz, tx_pos[2], params.map_origin[2]
    lam = C0 / f
    eta = eps_r - 1j * sigma / (EPS0 * 2 * math.pi * f)
    x0 = -params.nx * params.cell_size / 2

    def gain(X, Y):
        rho2 = X ** 2 + Y ** 2
        d1, d2 = rho2 + (ht - hr) ** 2, rho2 + (ht + hr) ** 2
        c = (ht + hr) / np.sqrt(d2)
        s = np.sqrt(eta - (1 - c * c))
        r_par = (eta * c - s) / (eta * c + s)
        return (lam / (4 * math.pi)) ** 2 * (1 / d1 + np.abs(r_par) ** 2 / d2)

    def rays(X, Y):
        rho2 = X ** 2 + Y ** 2
        return num_rays / (4 * math.pi) * ((ht - hr) / (rho2 + (ht - hr) ** 2) ** 1.5 +
                                           (ht + hr) / (rho2 + (ht + hr) ** 2) ** 1.5)

    c = params.cell_size
    return (cell_avg(gain, x0, x0, c, params.nx, params.ny),
            cell_avg(rays, x0, x0, c, params.nx, params.ny) * c * c)


def reciprocity_replicates(n0, reps):
    """Lattice sizes and seeds of the replicates of a reciprocity check.  The
    Fibonacci lattice is fixed in the global frame, so its per-cell counting
    error is deterministic for a given N; varying N (and the seed of the
    interaction choices) makes the replicates scatter by both errors, and
    their spread estimates the standard error of the mean."""
    return [(n0 + 7919 * r, r) for r in range(reps)]


def reciprocity_bound(a, b, cell, dist, z=4.5):
    """|mean_a - mean_b| allowed between the map value at B with the TX at A
    and at A with the TX at B.  a, b: replicate values.  Beyond z standard
    errors, the two cell averages differ at second order in cell/dist: one
    averages the gain over receiver positions around B, the other over
    transmitter positions around A (for a 1/d^2 gain each is within
    ~(cell/dist)^2 / 2 of the point value)."""
    a, b = np.asarray(a), np.asarray(b)
    se = math.hypot(a.std(ddof=1) / math.sqrt(len(a)), b.std(ddof=1) / math.sqrt(len(b)))
    return z * se + (cell / dist) ** 2 * max(a.mean(), b.mean())


RECIP_A = (0.0, 0.0, 10.0)
RECIP_PAIRS = [(9.0, 13.0, 1.5),     # same side as A: LoS, ground, wall, ground-wall, wall-ground
               (27.0, -6.0, 1.5)]    # behind the wall: transmission through the slab (R/T sampled)


def recip_scene():
    """Ground (half-space) and one 0.2 m slab wall at x = 20 m."""
    return S.ground_and_wall(wall_mat=(4.0, 0.02, 0.2))


def recip_params(rx, cell, deposit):
    """3 x 3 cells centred on rx (the centre cell is read), depth 2, 3.5 GHz."""
    return S.TraceParams(3.5e9, 2, cell_size=cell, nx=3, ny=3, map_origin=rx, deposit=deposit)
