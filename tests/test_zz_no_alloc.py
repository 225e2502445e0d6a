"""rm_radio_map_trace_noalloc: the entry point for callers that cannot
allocate device memory while they run (a serving loop with memory reserved
at start-up, an application that owns the GPU through its own pool, a thread
that must not wait on the allocator).  It must give the same maps and
counters as rm_radio_map_trace, call after call, from its static scratch."""
import ctypes as C

import numpy as np
import pytest
import torch

from synth import scenes as S
from gpu_helpers import FLOOR

pytestmark = pytest.mark.gpu


def _call(L, lib, gs, arr, ntx, prm, out):
    st = L.rm_stats()
    rc = lib.rm_radio_map_trace_noalloc(gs.handle, arr, ntx, C.byref(prm), C.c_void_p(out.data_ptr()),
                                        C.byref(st), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, st


def _same(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    mask = b > FLOOR
    assert mask.sum() > 1000
    # same rays and choices; only the order of the FP32 atomic additions differs
    assert np.all(np.abs(a - b)[mask] <= 2e-5 * b[mask])
    assert np.all(a[~mask] <= FLOOR)


def test_noalloc_matches_allocating_trace_twice(api):
    from paper_2504_21719_b300 import _lib as L
    lib = L.load()
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 10                                     # 1e6 rays of the 1e7-ray lattice
    gs = api.Scene.from_obj(sc)
    prm = api.params_from(p)
    arr = (L.rm_tx * 1)(api.tx_from(tx))
    ref = api.trace(gs, [tx], prm)
    out = torch.empty_like(ref["maps"])
    for _ in range(2):
        out.fill_(-1.0)                                    # the call must overwrite every cell
        rc, st = _call(L, lib, gs, arr, 1, prm, out)
        assert rc == L.RM_OK, lib.rm_last_error()
        torch.cuda.synchronize()
        _same(out, ref["maps"])
        assert st.rays == ref["stats"]["rays"] and st.segments == ref["stats"]["segments"]
        assert st.deposits == ref["stats"]["deposits"]
    gs.free()


def test_noalloc_batched_and_limits(api):
    from paper_2504_21719_b300 import _lib as L
    lib = L.load()
    sc, txs, p = S.workload(3)
    txs = txs[:5]
    for t in txs:
        t.ray_stride = 8
    gs = api.Scene.from_obj(sc)
    prm = api.params_from(p)
    arr = (L.rm_tx * len(txs))(*[api.tx_from(t) for t in txs])
    ref = api.trace(gs, txs, prm)
    out = torch.empty_like(ref["maps"])
    for _ in range(2):
        rc, st = _call(L, lib, gs, arr, len(txs), prm, out)
        assert rc == L.RM_OK, lib.rm_last_error()
        torch.cuda.synchronize()
        _same(out, ref["maps"])
        assert st.segments == ref["stats"]["segments"]
    # beyond the maximum: rejected on the host with a clear message
    big = (L.rm_tx * (L.RM_MAX_TX + 1))(*([api.tx_from(txs[0])] * (L.RM_MAX_TX + 1)))
    rc, _ = _call(L, lib, gs, big, L.RM_MAX_TX + 1, prm, out)
    assert rc == L.RM_EINVAL and b"ntx" in lib.rm_last_error()
    gs.free()


def test_noalloc_with_arrays(api):
    """A 200-element uniform linear array packs into 52 antenna-table records and
    fits the 16 KB static scratch; 600 irregular elements (600 records of 32 B)
    do not and are rejected on the host."""
    from paper_2504_21719_b300 import _lib as L
    lib = L.load()
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 50
    tx.ant_pos, tx.precoding = S.uniform_linear_array(200, p.freq_hz, 0.5, axis=1)
    gs = api.Scene.from_obj(sc)
    prm = api.params_from(p)
    arr, ntx = api._tx_array([tx])
    ref = api.trace(gs, [tx], prm)
    out = torch.empty_like(ref["maps"])
    rc, st = _call(L, lib, gs, arr, ntx, prm, out)
    assert rc == L.RM_OK, lib.rm_last_error()
    torch.cuda.synchronize()
    _same(out, ref["maps"])
    rng = np.random.default_rng(4)
    tx.ant_pos = rng.uniform(-0.05, 0.05, size=(600, 3))
    tx.precoding = np.ones(600) / np.sqrt(600.0)
    arr2, _ = api._tx_array([tx])
    rc, _ = _call(L, lib, gs, arr2, 1, prm, out)
    assert rc == L.RM_EINVAL and b"noalloc" in lib.rm_last_error()
    gs.free()
