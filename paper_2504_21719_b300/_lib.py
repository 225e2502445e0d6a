"""ctypes binding of librmsbr.so with the names of include/rmsbr.h.

Argument marshalling only: every step of the radio-map path runs in the CUDA
library.  Importing this module never falls back to anything else: if the
library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librmsbr.so")

RM_OK, RM_EINVAL, RM_ENOMEM, RM_ECUDA, RM_EOVERFLOW, RM_ETIMEOUT, RM_ESTATE = range(7)
STATUS_NAMES = ["RM_OK", "RM_EINVAL", "RM_ENOMEM", "RM_ECUDA", "RM_EOVERFLOW", "RM_ETIMEOUT", "RM_ESTATE"]
RM_MAX_DEPTH, RM_MAX_MATERIALS, RM_MAX_TX = 15, 32, 64
RM_REFLECT, RM_REFRACT, RM_LOS, RM_STATS, RM_DIFFUSE, RM_RECORD_COIN = 1, 2, 4, 8, 16, 32
RM_FAULT_ALLOC, RM_FAULT_LAUNCH, RM_FAULT_OVERFLOW = 1, 2, 3
NO_CELL = -32768
UINT64_MAX = (1 << 64) - 1


class rm_material(C.Structure):
    _fields_ = [("eps_r", C.c_float), ("sigma", C.c_float), ("thickness", C.c_float),
                ("scattering", C.c_float), ("xpd_k", C.c_float), ("pattern", C.c_int32),
                ("alpha_r", C.c_int32), ("alpha_i", C.c_int32), ("lobe_lambda", C.c_float)]


class rm_tx(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("yaw", C.c_float), ("pitch", C.c_float), ("roll", C.c_float),
                ("pol", C.c_int32), ("pattern", C.c_int32), ("num_rays", C.c_uint64),
                ("ray_begin", C.c_uint64), ("ray_count", C.c_uint64), ("ray_stride", C.c_uint64),
                ("seed", C.c_uint64), ("n_ant", C.c_int32), ("reserved", C.c_int32),
                ("ant_pos_host", C.c_void_p), ("precoding_host", C.c_void_p)]


class rm_trace_params(C.Structure):
    _fields_ = [("freq_hz", C.c_double), ("max_depth", C.c_int32), ("flags", C.c_uint32),
                ("map_origin", C.c_float * 3), ("cell_size", C.c_float), ("nx", C.c_int32),
                ("ny", C.c_int32), ("deposit", C.c_int32), ("block_size", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("queue_chunk", C.c_int32), ("rr_depth", C.c_int32),
                ("rr_max_prob", C.c_float), ("gain_threshold", C.c_float), ("refill_min", C.c_int32)]


_D = RM_MAX_DEPTH + 1


class rm_stats(C.Structure):
    _fields_ = [("rays", C.c_uint64), ("segments", C.c_uint64), ("nodes_visited", C.c_uint64),
                ("tris_tested", C.c_uint64), ("deposits", C.c_uint64), ("escapes", C.c_uint64),
                ("segments_per_depth", C.c_uint64 * _D), ("power_per_depth", C.c_double * _D),
                ("power2_per_depth", C.c_double * _D), ("escaped_power_per_depth", C.c_double * _D),
                ("status", C.c_int32), ("reserved", C.c_int32), ("kernel_ms", C.c_double)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if hasattr(v, "__len__") else v
        return out


class rm_segment_record(C.Structure):
    _fields_ = [("prim", C.c_int32), ("ix", C.c_int32), ("iy", C.c_int32), ("decision", C.c_int32)]


class rm_wedge(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("edge", C.c_float * 3), ("n0", C.c_float * 3), ("nn", C.c_float * 3),
                ("length", C.c_float), ("n", C.c_float), ("tri0", C.c_int32), ("trin", C.c_int32),
                ("mat0", C.c_int32), ("matn", C.c_int32)]


P = C.c_void_p
_SIGS = {
    "rm_scene_upload": ([P, C.c_int64, P, C.c_int64, P, P, C.c_int32, P, C.POINTER(P)], C.c_int),
    "rm_scene_upload_host": ([P, C.c_int64, P, C.c_int64, P, P, C.c_int32, P, C.POINTER(P)], C.c_int),
    "rm_scene_set_materials": ([P, P, C.c_int32, P], C.c_int),
    "rm_bvh_build": ([P, P], C.c_int),
    "rm_bvh_build_ex": ([P, C.c_int32, P], C.c_int),
    "rm_bvh_export": ([P, P, P, P, P], C.c_int),
    "rm_radio_map_trace": ([P, P, C.c_int32, P, P, P, P, P], C.c_int),
    "rm_radio_map_trace_mesh": ([P, P, P, C.c_int32, P, P, P, P, P], C.c_int),
    "rm_radio_map_grad": ([P, P, C.c_int32, P, P, P, P, P, P, P, P, P], C.c_int),
    "rm_radio_map_trace_hits": ([P, P, C.c_int32, P, P, P, C.c_uint64, P, P], C.c_int),
    "rm_radio_map_grad_hits": ([P, P, C.c_int32, P, P, P, C.c_uint64, P, P, P, P, P, P, P], C.c_int),
    "rm_radio_map_trace_mesh_hits": ([P, P, P, C.c_int32, P, P, P, C.c_uint64, P, P], C.c_int),
    "rm_radio_map_grad_mesh_hits": ([P, P, P, C.c_int32, P, P, P, C.c_uint64, P, P, P, P, P, P, P], C.c_int),
    "rm_radio_map_grad_mesh": ([P, P, P, C.c_int32, P, P, P, P, P, P, P, P, P], C.c_int),
    "rm_radio_map_trace_noalloc": ([P, P, C.c_int32, P, P, P, P], C.c_int),
    "rm_debug_array_factor": ([P, P, C.c_int32, P, P, P, C.c_uint64, P], C.c_int),
    "rm_db_mse_loss": ([P, P, C.c_int64, C.c_float, P, P, P, P], C.c_int),
    "rm_trace_plan_create": ([P, P, C.c_int32, P, P, P, C.POINTER(P)], C.c_int),
    "rm_trace_plan_launch": ([P, P], C.c_int),
    "rm_trace_plan_stats": ([P, P, P], C.c_int),
    "rm_trace_plan_free": ([P], None),
    "rm_scene_wedges": ([P, P, C.c_int64, P], C.c_int),
    "rm_diffraction_map": ([P, P, C.c_int64, P, C.c_int32, P, C.c_int64, P, P, P, P], C.c_int),
    "rm_diffraction_map_mesh": ([P, P, P, C.c_int64, P, C.c_int32, P, C.c_int64, P, P, P, P], C.c_int),
    "rm_scene_info": ([P, P, P, P, P], C.c_int),
    "rm_scene_free": ([P], None),
    "rm_last_error": ([], C.c_char_p),
    "rm_debug_inject": ([C.c_int32, C.c_int32], C.c_int),
    "rm_debug_alloc_count": ([], C.c_uint64),
    "rm_debug_fresnel_probe": ([P, C.c_double, P, C.c_int64, P, P, P], C.c_int),
    "rm_version": ([], C.c_char_p),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load librmsbr.so (raises OSError / RuntimeError if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2504_21719_b300.build.build() "
                               "(there is no fallback implementation)")
        lib = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def __getattr__(name):
    if name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)
