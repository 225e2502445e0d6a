"""FP64 CPU oracle for the SBR radio-map method (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package.  It wraps ``liboracle.so`` (``oracle.cpp``: plain C++17 + OpenMP,
FP64, brute-force intersection) with ctypes.  It shares no code with the CUDA
library; both read the same seeded scenes from ``synth``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.cpp")

F_REFLECT, F_REFRACT, F_LOS, F_DIFFUSE = 1, 2, 4, 16
NO_CELL = -32768


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++, -O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", _SO]
        subprocess.check_call(cmd)
    return _SO


class OrTx(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("yaw", C.c_double), ("pitch", C.c_double),
                ("roll", C.c_double), ("pol", C.c_int32), ("pattern", C.c_int32),
                ("num_rays", C.c_int64), ("ray_begin", C.c_int64), ("ray_count", C.c_int64),
                ("ray_stride", C.c_int64), ("seed", C.c_uint64), ("n_ant", C.c_int64),
                ("ant_pos", C.c_void_p), ("precoding", C.c_void_p)]


class OrParams(C.Structure):
    _fields_ = [("freq_hz", C.c_double), ("max_depth", C.c_int32), ("flags", C.c_int32),
                ("map_origin", C.c_double * 3), ("cell_size", C.c_double), ("nx", C.c_int32),
                ("ny", C.c_int32), ("deposit", C.c_int32), ("pad", C.c_int32),
                ("rr_depth", C.c_int32), ("pad2", C.c_int32), ("rr_max_prob", C.c_double),
                ("gain_threshold", C.c_double)]


class OrReport(C.Structure):
    _fields_ = [("segments", C.c_int64), ("deposits", C.c_int64), ("adopted_hit", C.c_int64),
                ("adopted_cell", C.c_int64), ("adopted_decision", C.c_int64),
                ("failures", C.c_int64), ("adopted_hit_tie", C.c_int64), ("fail_ray", C.c_int64),
                ("fail_depth", C.c_int32),
                ("fail_kind", C.c_int32), ("fail_info", C.c_double * 4),
                ("coin_checked", C.c_int64), ("coin_outside", C.c_int64), ("coin_max_dev", C.c_double),
                ("coin_max_ratio", C.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "fail_info"}
        d["fail_info"] = list(self.fail_info)
        return d


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.or_rng_u.restype = C.c_double
        _lib.or_rng_u.argtypes = [C.c_uint64, C.c_uint64, C.c_int]
        _lib.or_splitmix64.restype = C.c_uint64
        _lib.or_splitmix64.argtypes = [C.c_uint64]
        _lib.or_rng_diff.restype = C.c_double
        _lib.or_rng_diff.argtypes = [C.c_uint64, C.c_uint64, C.c_int, C.c_int]
        _lib.or_f_alpha.restype = C.c_double
        _lib.or_f_alpha.argtypes = [C.c_int, C.c_double]
        _lib.or_scat_pattern.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, P, P, P, C.c_int64, P]
        _lib.or_diffuse_dir.argtypes = [P, P, C.c_int64, P]
        _lib.or_wedges.restype = C.c_int64
        _lib.or_wedges.argtypes = [P, C.c_int64, P, C.c_int64, P, P, C.c_int64]
        _lib.or_utd_F.argtypes = [C.c_double, P]
        _lib.or_utd_field.argtypes = [P, P, P, P, C.c_double, P, P, C.c_double, P]
        _lib.or_diffraction_point.restype = C.c_int
        _lib.or_diffraction_point.argtypes = [P, P, C.c_double, C.c_double, C.c_double, P]
        _lib.or_diffraction_map.restype = C.c_int
        _lib.or_diffraction_map.argtypes = [P, C.c_int64, P, C.c_int64, P, P, C.c_int, P, P, C.c_int64, C.c_int,
                                            P, C.c_int64, P, P, P, P, P, C.c_int64]
        _lib.or_diffuse_interact.argtypes = [P, P, P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                             C.c_double, C.c_int, C.c_int, C.c_int, C.c_double, P, P, P]
        _lib.or_fibonacci.argtypes = [C.c_int64, C.c_int64, C.c_int64, C.c_int64, P]
        _lib.or_tx_field.argtypes = [P, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int,
                                     C.c_int, P]
        _lib.or_rotation.argtypes = [C.c_double, C.c_double, C.c_double, P]
        _lib.or_csqrt.argtypes = [C.c_double, C.c_double, P]
        _lib.or_fresnel.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, P]
        _lib.or_fresnel_vac_t.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, P]
        _lib.or_interact.argtypes = [P, P, P, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.c_int, P, P]
        _lib.or_closest_hit.argtypes = [P, C.c_int64, P, C.c_int64, P, P, C.c_int64, P, P, P]
        _lib.or_radio_map.restype = C.c_int
        _lib.or_radio_map.argtypes = [P, C.c_int64, P, C.c_int64, P, P, C.c_int, P, P, P, C.c_int, P,
                                      P, P, P, P, P, P]
        _lib.or_grad.restype = C.c_int
        _lib.or_grad.argtypes = [P, C.c_int64, P, C.c_int64, P, P, C.c_int, P, P, P, P, P, P]
        _lib.or_branch_all.restype = C.c_int
        _lib.or_branch_all.argtypes = [P, C.c_int64, P, C.c_int64, P, P, C.c_int, P, P, P, P, P]
        _lib.or_morton.argtypes = [P, P, C.c_int64, P, P, P]
        _lib.or_lbvh.restype = C.c_int
        _lib.or_lbvh.argtypes = [P, P, C.c_int64, P, P, P, P, P]
        _lib.or_sah_bvh.restype = C.c_int
        _lib.or_sah_bvh.argtypes = [P, P, C.c_int64, P, P, P, P, P]
        _lib.or_num_threads.restype = C.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(lib().or_num_threads())


# ----------------------------------------------------------------------------
# conversions from the synth dataclasses
# ----------------------------------------------------------------------------

def make_tx(tx) -> OrTx:
    t = OrTx()
    for i in range(3):
        t.pos[i] = float(tx.pos[i])
    t.yaw, t.pitch, t.roll = float(tx.yaw), float(tx.pitch), float(tx.roll)
    t.pol, t.pattern = int(tx.pol), int(tx.pattern)
    t.num_rays, t.ray_begin = int(tx.num_rays), int(tx.ray_begin)
    t.ray_count, t.ray_stride = int(tx.ray_count), int(tx.ray_stride)
    t.seed = int(tx.seed)
    ant = getattr(tx, "ant_pos", None)
    if ant is not None and len(ant):
        a = np.ascontiguousarray(ant, np.float64).reshape(-1, 3)
        pre = np.asarray(tx.precoding, np.complex128).reshape(-1)
        pc = np.ascontiguousarray(np.stack([pre.real, pre.imag], 1), np.float64)
        t._keep = (a, pc)  # keep the buffers alive with the struct
        t.n_ant = len(a)
        t.ant_pos = a.ctypes.data
        t.precoding = pc.ctypes.data
    return t


def make_params(p) -> OrParams:
    q = OrParams()
    q.freq_hz = float(p.freq_hz)
    q.max_depth = int(p.max_depth)
    q.flags = (F_REFLECT if p.reflect else 0) | (F_REFRACT if p.refract else 0) | (F_LOS if p.los else 0)
    if getattr(p, "diffuse", False):
        q.flags |= F_DIFFUSE
    for i in range(3):
        q.map_origin[i] = float(p.map_origin[i])
    q.cell_size = float(p.cell_size)
    q.nx, q.ny, q.deposit = int(p.nx), int(p.ny), int(p.deposit)
    q.rr_depth = int(getattr(p, "rr_depth", 0))
    q.rr_max_prob = float(getattr(p, "rr_max_prob", 0.0))
    q.gain_threshold = float(getattr(p, "gain_threshold", 0.0))
    return q


def _scene_arrays(scene):
    v = np.ascontiguousarray(scene.verts, np.float32)
    t = np.ascontiguousarray(scene.tris, np.int32)
    m = np.ascontiguousarray(scene.tri_mat, np.int32)
    mats = np.ascontiguousarray(scene.mats, np.float32)
    return v, t, m, mats


def _scat(scene):
    sc = getattr(scene, "scat", None)
    return None if sc is None else np.ascontiguousarray(sc, np.float32).reshape(-1, 6)


# ----------------------------------------------------------------------------
# elementary functions (for the pins)
# ----------------------------------------------------------------------------

def rng_u(seed: int, n: int, l: int) -> float:
    return float(lib().or_rng_u(seed, n, l))


def splitmix64(x: int) -> int:
    return int(lib().or_splitmix64(x))


def rng_diff(seed: int, n: int, l: int, j: int) -> float:
    """Variate j (0, 1: direction; 2, 3: phases) of a diffuse reflection."""
    return float(lib().or_rng_diff(seed, n, l, j))


def f_alpha(alpha: int, cos_i: float) -> float:
    return float(lib().or_f_alpha(alpha, cos_i))


def scat_pattern(pattern, ki, n, ks, alpha_r=1, alpha_i=1, lam=1.0):
    """f_s(k_i, k_s, n) for directions ks [m, 3]."""
    ki = np.ascontiguousarray(ki, np.float64)
    n = np.ascontiguousarray(n, np.float64)
    ks = np.ascontiguousarray(ks, np.float64).reshape(-1, 3)
    out = np.empty(len(ks), np.float64)
    lib().or_scat_pattern(int(pattern), int(alpha_r), int(alpha_i), float(lam), _p(ki), _p(n), _p(ks), len(ks),
                          _p(out))
    return out


def diffuse_dir(n, u):
    """Scattered directions for variate pairs u [m, 2] about the normal n."""
    n = np.ascontiguousarray(n, np.float64)
    u = np.ascontiguousarray(u, np.float64).reshape(-1, 2)
    out = np.empty((len(u), 3), np.float64)
    lib().or_diffuse_dir(_p(n), _p(u), len(u), _p(out))
    return out


def fibonacci(N: int, begin: int = 0, count: int | None = None, stride: int = 1) -> np.ndarray:
    if count is None:
        count = (N - begin + stride - 1) // stride
    out = np.empty((count, 3), np.float64)
    lib().or_fibonacci(N, begin, count, stride, _p(out))
    return out


def tx_field(dirs, yaw=0.0, pitch=0.0, roll=0.0, pattern=0, pol=0) -> np.ndarray:
    d = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    out = np.empty_like(d)
    lib().or_tx_field(_p(d), len(d), yaw, pitch, roll, pattern, pol, _p(out))
    return out


def rotation(yaw, pitch, roll) -> np.ndarray:
    out = np.empty(9, np.float64)
    lib().or_rotation(yaw, pitch, roll, _p(out))
    return out.reshape(3, 3)


def csqrt(z: complex) -> complex:
    out = np.empty(2, np.float64)
    lib().or_csqrt(z.real, z.imag, _p(out))
    return complex(out[0], out[1])


def fresnel(eps_r, sigma, freq_hz, cos1, thickness=0.0):
    """(r_perp, r_par, t_perp, t_par) for a half-space (thickness <= 0) or slab."""
    omega = 2 * np.pi * freq_hz
    k0d = omega / 299792458.0 * thickness if thickness > 0 else 0.0
    out = np.empty(8, np.float64)
    lib().or_fresnel(eps_r, sigma, omega, cos1, k0d, _p(out))
    return tuple(complex(out[2 * i], out[2 * i + 1]) for i in range(4))


def fresnel_vac_t(eps_r, sigma, freq_hz, cos1):
    out = np.empty(4, np.float64)
    lib().or_fresnel_vac_t(eps_r, sigma, 2 * np.pi * freq_hz, cos1, _p(out))
    return complex(out[0], out[1]), complex(out[2], out[3])


def interact(k, n, E, eps_r, sigma, freq_hz, thickness, dec):
    k = np.ascontiguousarray(k, np.float64)
    n = np.ascontiguousarray(n, np.float64)
    E = np.asarray(E, np.complex128)
    e6 = np.ascontiguousarray(np.stack([E.real, E.imag], 1).reshape(-1), np.float64)
    omega = 2 * np.pi * freq_hz
    k0d = omega / 299792458.0 * thickness if thickness > 0 else 0.0
    ko = np.empty(3, np.float64)
    eo = np.empty(6, np.float64)
    lib().or_interact(_p(k), _p(n), _p(e6), eps_r, sigma, omega, k0d, dec, _p(ko), _p(eo))
    return ko, eo[0::2] + 1j * eo[1::2]


def diffuse_interact(k, n, E, eps_r, sigma, freq_hz, thickness, S, K_x=0.0, pattern=0, alpha_r=1, alpha_i=1,
                     lam=1.0, u=(0.3, 0.2, 0.0, 0.0)):
    """One diffuse reflection: (scattered direction, field)."""
    k = np.ascontiguousarray(k, np.float64)
    n = np.ascontiguousarray(n, np.float64)
    E = np.asarray(E, np.complex128)
    e6 = np.ascontiguousarray(np.stack([E.real, E.imag], 1).reshape(-1), np.float64)
    omega = 2 * np.pi * freq_hz
    k0d = omega / 299792458.0 * thickness if thickness > 0 else 0.0
    u4 = np.ascontiguousarray(u, np.float64)
    ko = np.empty(3, np.float64)
    eo = np.empty(6, np.float64)
    lib().or_diffuse_interact(_p(k), _p(n), _p(e6), eps_r, sigma, omega, k0d, S, K_x, int(pattern), int(alpha_r),
                              int(alpha_i), lam, _p(u4), _p(ko), _p(eo))
    return ko, eo[0::2] + 1j * eo[1::2]


def closest_hit(scene, o, k, exclude=None):
    v, t, _, _ = _scene_arrays(scene)
    o = np.ascontiguousarray(o, np.float64).reshape(-1, 3)
    k = np.ascontiguousarray(k, np.float64).reshape(-1, 3)
    ex = None if exclude is None else np.ascontiguousarray(exclude, np.int32)
    prim = np.empty(len(o), np.int32)
    tt = np.empty(len(o), np.float64)
    lib().or_closest_hit(_p(v), len(v), _p(t), len(t), _p(o), _p(k), len(o), _p(ex), _p(prim), _p(tt))
    return prim, tt


# ----------------------------------------------------------------------------
# radio maps
# ----------------------------------------------------------------------------
MODES = {"plain": 0, "replay": 1, "frozen": 2}


def radio_map(scene, tx, params, mode: str = "plain", record=None, want_record: bool = False,
              sampling_mats=None, eval_mats=None, stats: bool = False, mass: bool = False):
    """Radio map [ny, nx] (float64) of one transmitter.

    mode 'plain'  : decisions from the counter-based RNG; ``want_record``
                    returns the per-segment record int32 [count, L+1, 4].
    mode 'replay' : ``record`` is the GPU's record; every differing discrete
                    choice must be an FP64-certified near-tie (see report).
    mode 'frozen' : hits, cells and decisions are taken from ``record``.
    """
    v, t, m, mats = _scene_arrays(scene)
    otx, op = make_tx(tx), make_params(params)
    L = int(params.max_depth)
    cnt = tx.count()
    rec = None
    if mode in ("replay", "frozen"):
        rec = np.ascontiguousarray(record, np.int32).reshape(cnt, L + 1, 4)
        if mode == "replay":
            rec = rec.copy()
    elif want_record:
        rec = np.zeros((cnt, L + 1, 4), np.int32)
    sm = None if sampling_mats is None else np.ascontiguousarray(np.asarray(sampling_mats, np.float64)[:, :2])
    em = None if eval_mats is None else np.ascontiguousarray(np.asarray(eval_mats, np.float64)[:, :2])
    mp = np.empty((params.ny, params.nx), np.float64)
    st = np.empty(3 * (L + 1), np.float64) if stats else None
    ms = np.empty((3, params.ny, params.nx), np.float64) if mass else None
    rep = OrReport()
    sc = _scat(scene)
    rc = lib().or_radio_map(_p(v), len(v), _p(t), len(t), _p(m), _p(mats), len(mats), _p(sc), C.byref(otx),
                            C.byref(op), MODES[mode], _p(rec), _p(sm), _p(em), _p(mp), _p(st),
                            C.byref(rep), _p(ms))
    if rc != 0:
        raise ValueError(f"or_radio_map failed ({rc})")
    out = {"map": mp}
    if want_record or mode != "plain":
        out["record"] = rec
    if stats:
        s = st.reshape(3, L + 1)
        out["power"], out["power2"], out["escaped"] = s[0], s[1], s[2]
    if mode == "replay":
        out["report"] = rep.as_dict()
    if mass:
        out["mass"], out["cmass"], out["amass"] = ms[0], ms[1], ms[2]
    return out


def radio_map_mesh(scene, tx, params, surf_verts, surf_tris, mode: str = "plain", record=None,
                   want_record: bool = False, slack: bool = False):
    """Radio map on a mesh measurement surface: [n_surf] (float64), one cell per
    surface triangle.  params' map geometry is unused; mode 'plain' or 'replay'
    as in radio_map.  ``slack`` returns, per cell, the values of the crossings
    within tol of its boundary or of a window end."""
    v, t, m, mats = _scene_arrays(scene)
    sv = np.ascontiguousarray(surf_verts, np.float32)
    st_ = np.ascontiguousarray(surf_tris, np.int32)
    otx, op = make_tx(tx), make_params(params)
    L = int(params.max_depth)
    cnt = tx.count()
    rec = None
    if mode == "replay":
        rec = np.ascontiguousarray(record, np.int32).reshape(cnt, L + 1, 4).copy()
    elif mode != "plain":
        raise ValueError("mode must be 'plain' or 'replay'")
    elif want_record:
        rec = np.zeros((cnt, L + 1, 4), np.int32)
    mp = np.empty(len(st_), np.float64)
    sl = np.empty(len(st_), np.float64) if slack else None
    rep = OrReport()
    sc = _scat(scene)
    rc = lib().or_radio_map_mesh(_p(v), len(v), _p(t), len(t), _p(m), _p(mats), len(mats), _p(sc), C.byref(otx),
                                 C.byref(op), _p(sv), _p(st_), C.c_int64(len(st_)), MODES[mode], _p(rec), _p(mp), _p(sl),
                                 C.byref(rep))
    if rc != 0:
        raise ValueError(f"or_radio_map_mesh failed ({rc})")
    out = {"map": mp}
    if want_record or mode != "plain":
        out["record"] = rec
    if mode == "replay":
        out["report"] = rep.as_dict()
    if slack:
        out["slack"] = sl
    return out


def grad_mesh(scene, tx, params, surf_verts, surf_tris, record, dLdC):
    """d/d(eps_r, sigma, tx xyz) of sum(dLdC * C) for a map on a mesh measurement
    surface (dLdC [n_surf]), along the record's frozen hits and decisions."""
    v, t, m, mats = _scene_arrays(scene)
    sv = np.ascontiguousarray(surf_verts, np.float32)
    st_ = np.ascontiguousarray(surf_tris, np.int32)
    otx, op = make_tx(tx), make_params(params)
    rec = np.ascontiguousarray(record, np.int32)
    g = np.ascontiguousarray(dLdC, np.float64).reshape(-1)
    if len(g) != len(st_):
        raise ValueError("dLdC must have one value per surface triangle")
    nm = len(mats)
    out = np.empty(2 * nm + 3, np.float64)
    sc = _scat(scene)
    rc = lib().or_grad_mesh(_p(v), len(v), _p(t), len(t), _p(m), _p(mats), nm, _p(sc), C.byref(otx), C.byref(op),
                            _p(sv), _p(st_), C.c_int64(len(st_)), _p(rec), _p(g), _p(out))
    if rc != 0:
        raise ValueError(f"or_grad_mesh failed ({rc}): at most 8 materials, valid scattering parameters")
    return out[:nm].copy(), out[nm:2 * nm].copy(), out[2 * nm:].copy()


def grad(scene, tx, params, record, dLdC):
    """d/d(eps_r, sigma, tx xyz) of sum(dLdC * C) with frozen choices (dual numbers)."""
    v, t, m, mats = _scene_arrays(scene)
    otx, op = make_tx(tx), make_params(params)
    rec = np.ascontiguousarray(record, np.int32)
    g = np.ascontiguousarray(dLdC, np.float64)
    nm = len(mats)
    out = np.empty(2 * nm + 3, np.float64)
    sc = _scat(scene)
    rc = lib().or_grad(_p(v), len(v), _p(t), len(t), _p(m), _p(mats), nm, _p(sc), C.byref(otx), C.byref(op),
                       _p(rec), _p(g), _p(out))
    if rc != 0:
        raise ValueError(f"or_grad failed ({rc}): at most 8 materials, valid scattering parameters")
    return out[:nm].copy(), out[nm:2 * nm].copy(), out[2 * nm:].copy()


def branch_all(scene, tx, params):
    """Exact expectation over interaction choices: (map, power[l], escaped[l])."""
    v, t, m, mats = _scene_arrays(scene)
    otx, op = make_tx(tx), make_params(params)
    L = int(params.max_depth)
    mp = np.empty((params.ny, params.nx), np.float64)
    pw = np.empty(L + 1, np.float64)
    es = np.empty(L + 1, np.float64)
    rc = lib().or_branch_all(_p(v), len(v), _p(t), len(t), _p(m), _p(mats), len(mats), C.byref(otx),
                             C.byref(op), _p(mp), _p(pw), _p(es))
    if rc != 0:
        raise ValueError(f"or_branch_all failed ({rc}): depth too large or diffuse reflection on")
    return mp, pw, es


def morton(scene):
    """(keys [nt] with 2^64-1 for large triangles, AABBs [nt, 6], number of large triangles)."""
    v, t, _, _ = _scene_arrays(scene)
    keys = np.empty(len(t), np.uint64)
    box = np.empty((len(t), 6), np.float32)
    nl = C.c_int64(0)
    lib().or_morton(_p(v), _p(t), len(t), _p(keys), _p(box), C.byref(nl))
    return keys, box, int(nl.value)


def lbvh(scene):
    """Reference LBVH: sorted keys, order, nlarge, child [ns-1, 2], child AABBs [ns-1, 2, 6]
    with ns = nt - nlarge (the large triangles are the last nlarge entries of order)."""
    return _tree(scene, lib().or_lbvh)


def sah_bvh(scene):
    """Reference binned-SAH tree over the same leaves as ``lbvh`` (32 centroid bins
    per axis, stable partitions from the Morton order, node i numbered by its
    split position, root 0); keys[p] is the Morton key of the triangle at p."""
    return _tree(scene, lib().or_sah_bvh)


def _tree(scene, fn):
    v, t, _, _ = _scene_arrays(scene)
    nt = len(t)
    keys = np.zeros(max(nt, 1), np.uint64)
    order = np.zeros(max(nt, 1), np.int32)
    child = np.zeros((max(nt - 1, 1), 2), np.int32)
    box = np.zeros((max(nt - 1, 1), 2, 6), np.float32)
    nl = C.c_int64(0)
    fn(_p(v), _p(t), nt, _p(keys), _p(order), _p(child), _p(box), C.byref(nl))
    ns = nt - int(nl.value)
    return {"keys": keys[:nt], "order": order[:nt], "nlarge": int(nl.value), "child": child[:max(ns - 1, 0)],
            "child_aabb": box[:max(ns - 1, 0)]}


# ----------------------------------------------------------------------------
# first-order diffraction radio map
# ----------------------------------------------------------------------------

def wedges(scene) -> np.ndarray:
    """[nw, 16] = o(3) e(3) n0(3) nn(3) length n tri0 trin, ordered by (tri0, trin)."""
    v, t, m, _ = _scene_arrays(scene)
    n = lib().or_wedges(_p(v), len(v), _p(t), len(t), _p(m), None, 0)
    out = np.zeros((max(n, 1), 16), np.float64)
    lib().or_wedges(_p(v), len(v), _p(t), len(t), _p(m), _p(out), n)
    return out[:n]


def utd_F(x: float) -> complex:
    out = np.empty(2, np.float64)
    lib().or_utd_F(float(x), _p(out))
    return complex(out[0], out[1])


def utd_field(wedge16, s, v, sd, sobs, E, mats=((3.0, 0.0), (3.0, 0.0)), freq_hz=3.5e9):
    """(E_d,phi, E_d,beta0) of one incident field E (3 complex) for the pins."""
    w = np.ascontiguousarray(wedge16, np.float64)
    E = np.asarray(E, np.complex128)
    e6 = np.ascontiguousarray(np.stack([E.real, E.imag], 1).reshape(-1), np.float64)
    m4 = np.ascontiguousarray(np.asarray(mats, np.float64).reshape(-1))
    out = np.empty(4, np.float64)
    lib().or_utd_field(_p(w), _p(np.ascontiguousarray(s, np.float64)), _p(np.ascontiguousarray(v, np.float64)),
                       _p(np.ascontiguousarray(sd, np.float64)), float(sobs), _p(e6), _p(m4),
                       2 * np.pi * freq_hz, _p(out))
    return complex(out[0], out[1]), complex(out[2], out[3])


def diffraction_point(wedge16, s, x, phi, zM):
    """(t [3], weighting factor |dt/dx x dt/dphi|) or None when the ray misses the plane."""
    out = np.empty(4, np.float64)
    ok = lib().or_diffraction_point(_p(np.ascontiguousarray(wedge16, np.float64)),
                                    _p(np.ascontiguousarray(s, np.float64)), float(x), float(phi), float(zM), _p(out))
    return (out[:3].copy(), float(out[3])) if ok else None


def diffraction_map(scene, tx, params, samples_per_wedge: int, mode: str = "plain", record=None,
                    want_record: bool = False, slack: bool = False, wedge_index=None):
    """First-order diffraction map [ny, nx] of one transmitter (oracle); with
    ``slack`` also the per-cell value change of the deposits under a +-1e-5 rad
    shift of their Keller azimuth.  ``wedge_index``: positions in wedges(scene)
    of the wedges to sample (default: all); the record follows that list."""
    v, t, m, mats = _scene_arrays(scene)
    otx, op = make_tx(tx), make_params(params)
    sel = None
    if wedge_index is not None:
        sel = np.ascontiguousarray(wedge_index, np.int64)
        nw = len(sel)
    else:
        nw = len(wedges(scene))
    rec = None
    if mode == "replay":
        rec = np.ascontiguousarray(record, np.int32).reshape(nw * samples_per_wedge, 4).copy()
    elif want_record:
        rec = np.zeros((nw * samples_per_wedge, 4), np.int32)
    mp = np.empty((params.ny, params.nx), np.float64)
    sl = np.empty((params.ny, params.nx), np.float64) if slack else None
    cnt = np.empty(3, np.float64)
    rep = OrReport()
    rc = lib().or_diffraction_map(_p(v), len(v), _p(t), len(t), _p(m), _p(mats), len(mats), C.byref(otx),
                                  C.byref(op), int(samples_per_wedge), {"plain": 0, "replay": 1}[mode], _p(rec),
                                  0 if rec is None else len(rec), _p(mp), _p(cnt), C.byref(rep), _p(sl), _p(sel),
                                  0 if sel is None else len(sel))
    if rc != 0:
        raise ValueError(f"or_diffraction_map failed ({rc})")
    out = {"map": mp, "crossings": int(cnt[0]), "visible": int(cnt[1]), "wedges": int(cnt[2])}
    if rec is not None:
        out["record"] = rec
    if mode == "replay":
        out["report"] = rep.as_dict()
    if slack:
        out["slack"] = sl
    return out


def diffraction_map_mesh(scene, tx, params, samples_per_wedge: int, surf_verts, surf_tris, mode: str = "plain",
                         record=None, want_record: bool = False, slack: bool = False, wedge_index=None):
    """Diffraction map on a mesh measurement surface: [n_surf] (float64).  Record
    [nw * N', 4] = {incident bit (-2 source behind both faces), crossings, 0, 0};
    replay certifies the incident bit only.  ``wedge_index``: positions in
    wedges(scene) of the wedges to sample (default: all); the record follows it."""
    v, t, m, mats = _scene_arrays(scene)
    sv = np.ascontiguousarray(surf_verts, np.float32)
    st_ = np.ascontiguousarray(surf_tris, np.int32)
    otx, op = make_tx(tx), make_params(params)
    sel = None
    if wedge_index is not None:
        sel = np.ascontiguousarray(wedge_index, np.int64)
        nw = len(sel)
    else:
        nw = len(wedges(scene))
    n = nw * int(samples_per_wedge)
    rec = None
    if mode == "replay":
        rec = np.ascontiguousarray(record, np.int32).reshape(n, 4).copy()
    elif want_record:
        rec = np.zeros((max(n, 1), 4), np.int32)
    mp = np.empty(len(st_), np.float64)
    sl = np.empty(len(st_), np.float64) if slack else None
    rep = OrReport()
    rc = lib().or_diffraction_map_mesh(_p(v), len(v), _p(t), len(t), _p(m), _p(mats), len(mats), C.byref(otx),
                                       C.byref(op), C.c_int64(int(samples_per_wedge)), _p(sv), _p(st_),
                                       C.c_int64(len(st_)), MODES[mode], _p(rec), C.c_int64(max(n, 1)), _p(mp),
                                       _p(sl), C.byref(rep), _p(sel), C.c_int64(0 if sel is None else len(sel)))
    if rc != 0:
        raise ValueError(f"or_diffraction_map_mesh failed ({rc})")
    out = {"map": mp, "wedges": nw}
    if want_record or mode != "plain":
        out["record"] = rec
    if mode == "replay":
        out["report"] = rep.as_dict()
    if slack:
        out["slack"] = sl
    return out
