"""The C-ABI library builds, loads, exports every entry point declared in
include/rmsbr.h with matching struct layouts, and rejects bad arguments on
the host (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rmsbr.h")


@pytest.fixture(scope="module")
def L():
    from paper_2504_21719_b300 import build
    build.build()
    from paper_2504_21719_b300 import _lib
    _lib.load()
    return _lib


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rm_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 14
    lib = L.load()
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.check_output(["nm", "-D", "--defined-only", L.LIB_PATH]).decode()
    exported = set(re.findall(r" T (rm_\w+)", out))
    assert set(names) <= exported
    assert set(names) == set(L._SIGS)


def test_struct_layouts_match_header(L, tmp_path):
    fields = {
        "rm_material": ["eps_r", "sigma", "thickness", "scattering", "xpd_k", "pattern", "alpha_r", "alpha_i",
                        "lobe_lambda"],
        "rm_tx": ["pos", "yaw", "pol", "pattern", "num_rays", "ray_begin", "ray_count", "ray_stride", "seed",
                  "n_ant", "ant_pos_host", "precoding_host"],
        "rm_trace_params": ["freq_hz", "max_depth", "flags", "map_origin", "cell_size", "nx", "ny", "deposit",
                            "block_size", "blocks_per_sm", "queue_chunk", "rr_depth", "rr_max_prob",
                            "gain_threshold", "refill_min"],
        "rm_stats": ["rays", "segments", "escapes", "segments_per_depth", "power_per_depth", "power2_per_depth",
                     "escaped_power_per_depth", "status", "kernel_ms"],
        "rm_segment_record": ["prim", "ix", "iy", "decision"],
        "rm_wedge": ["origin", "edge", "n0", "nn", "length", "n", "tri0", "trin", "mat0", "matn"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rmsbr.h"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(c), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for s, fs in fields.items():
        cls = getattr(L, s)
        assert int(got[s]) == C.sizeof(cls), s
        for f in fs:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


def test_host_validation_without_gpu(L):
    lib = L.load()
    h = C.c_void_p()
    # no materials -> RM_EINVAL before any CUDA call
    assert lib.rm_scene_upload(None, 0, None, 0, None, None, 0, None, C.byref(h)) == L.RM_EINVAL
    assert b"nm" in lib.rm_last_error()
    bad = (L.rm_material * 1)(L.rm_material(-1.0, 0.0, 0.0))
    assert lib.rm_scene_upload(None, 0, None, 0, None, bad, 1, None, C.byref(h)) == L.RM_EINVAL
    # diffuse parameters: S outside [0, 1], an unknown pattern, alpha out of range
    for kw in (dict(scattering=1.5), dict(scattering=0.5, pattern=3), dict(scattering=0.5, pattern=1, alpha_r=0),
               dict(scattering=0.5, pattern=2, alpha_r=2, alpha_i=40, lobe_lambda=0.5),
               dict(scattering=0.5, xpd_k=-0.2)):
        m = L.rm_material(4.0, 0.01, 0.2)
        for k, v in kw.items():
            setattr(m, k, v)
        assert lib.rm_scene_upload(None, 0, None, 0, None, (L.rm_material * 1)(m), 1, None, C.byref(h)) == L.RM_EINVAL
        assert b"material 0" in lib.rm_last_error()
    # host upload: index ranges are checked on the host, before any CUDA call
    import numpy as np
    good = (L.rm_material * 1)(L.rm_material(4.0, 0.01, 0.2))
    v = np.zeros((3, 3), np.float32)
    for t, m in ((np.array([[0, 1, 3]], np.int32), np.zeros(1, np.int32)),
                 (np.array([[0, -1, 2]], np.int32), np.zeros(1, np.int32)),
                 (np.array([[0, 1, 2]], np.int32), np.ones(1, np.int32))):
        assert lib.rm_scene_upload_host(v.ctypes.data, 3, t.ctypes.data, 1, m.ctypes.data, good, 1, None,
                                        C.byref(h)) == L.RM_EINVAL
        assert b"out of range" in lib.rm_last_error()
    assert lib.rm_scene_upload_host(None, 0, None, 1, None, good, 1, None, C.byref(h)) == L.RM_EINVAL
    assert lib.rm_radio_map_trace(None, None, 1, None, None, None, None, None) == L.RM_EINVAL
    assert lib.rm_radio_map_grad(None, None, 1, None, None, None, None, None, None, None, None, None) == L.RM_EINVAL
    assert lib.rm_db_mse_loss(None, None, 10, 0.0, None, None, None, None) == L.RM_EINVAL
    n = C.c_int64()
    assert lib.rm_scene_wedges(None, None, 0, C.byref(n)) == L.RM_EINVAL
    assert lib.rm_diffraction_map(None, None, 0, None, 1, None, 16, None, None, None, None) == L.RM_EINVAL
    assert lib.rm_trace_plan_launch(None, None) == L.RM_EINVAL
    assert lib.rm_radio_map_trace_mesh(None, None, None, 1, None, None, None, None, None) == L.RM_EINVAL
    assert lib.rm_radio_map_grad_mesh(None, None, None, 1, None, None, None, None, None, None, None, None,
                                      None) == L.RM_EINVAL
    assert b"surface" in lib.rm_last_error()
    assert lib.rm_bvh_build(None, None) == L.RM_EINVAL
    assert lib.rm_scene_info(None, None, None, None, None) == L.RM_EINVAL
    lib.rm_scene_free(None)
    lib.rm_trace_plan_free(None)
    assert lib.rm_version().startswith(b"rmsbr")


def test_no_fallback_when_library_missing(L, tmp_path):
    from paper_2504_21719_b300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def test_tx_array_keeps_antenna_buffers_alive(L):
    """The rm_tx copies handed to the library point at the binding's antenna
    buffers (double positions and precoding); those must outlive the
    temporary structs the binding builds from user objects."""
    import gc

    import numpy as np

    from paper_2504_21719_b300 import api
    from synth import scenes as S
    tx = S.Tx(pos=(0.0, 0.0, 20.0), num_rays=1000, seed=1)
    tx.ant_pos, tx.precoding = S.uniform_linear_array(1024, 3.5e9, 0.5)
    arr, n = api._tx_array([tx])
    gc.collect()
    junk = [np.full(2048, 7.0) for _ in range(64)]  # reuse freed blocks, if any
    t = arr[0]
    assert n == 1 and t.n_ant == 1024
    pos = np.ctypeslib.as_array(C.cast(t.ant_pos_host, C.POINTER(C.c_double)), shape=(1024, 3))
    pre = np.ctypeslib.as_array(C.cast(t.precoding_host, C.POINTER(C.c_double)), shape=(1024, 2))
    assert np.array_equal(pos, tx.ant_pos)
    assert np.array_equal(pre[:, 0] + 1j * pre[:, 1], tx.precoding)
    del junk
