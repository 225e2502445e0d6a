"""rm_radio_map_trace_noalloc: the entry point for callers that cannot
allocate device memory while they run (a serving loop with memory reserved
at start-up, an application that owns the GPU through its own pool, a thread
that must not wait on the allocator).  It must give the same maps and
counters as rm_radio_map_trace, call after call, from its static scratch,
and it must make no allocation at all."""
import ctypes as C
import threading

import numpy as np
import pytest
import torch

from synth import scenes as S
from gpu_helpers import FLOOR

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24          # FP32 unit roundoff


def _call(L, lib, gs, arr, ntx, prm, out, stream=None):
    st = L.rm_stats()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.rm_radio_map_trace_noalloc(gs.handle, arr, ntx, C.byref(prm), C.c_void_p(out.data_ptr()),
                                        C.byref(st), C.c_void_p(s.cuda_stream))
    return rc, st


def _deposit_counts(rec, txs, L, ny, nx):
    """Deposits per cell from a (box-deposit) record [.., 4] = {prim, ix, iy, decision}:
    count x (L + 1) records of each transmitter, one transmitter after the other."""
    r = rec.view(-1, 4)
    out = torch.zeros((len(txs), ny * nx), dtype=torch.float64, device=rec.device)
    b = 0
    for t, tx in enumerate(txs):
        e = b + tx.count() * (L + 1)
        ix, iy = r[b:e, 1].long(), r[b:e, 2].long()
        ok = (ix >= 0) & (ix < nx) & (iy >= 0) & (iy < ny)
        out[t] += torch.bincount((iy * nx + ix)[ok], minlength=ny * nx).double()
        b = e
    assert b == r.shape[0]
    return out.view(len(txs), ny, nx)


def _same(a, b, counts):
    """a: noalloc map (FP32 sums of the deposits in atomic order); b: the
    allocating trace's map (FP64 sums rounded once to FP32).  Summing n
    positive FP32 terms in any order errs by at most (n - 1) u of the exact
    sum; the reference adds one rounding.  The bound per cell is therefore
    (n + 1) u (1 + 2 u n) relative, n = that cell's deposit count."""
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    n = counts.cpu().numpy()
    mask = b > FLOOR
    assert mask.sum() > 1000
    bound = (n + 1.0) * U32 * (1.0 + 2.0 * U32 * n) * b
    assert np.all(np.abs(a - b)[mask] <= bound[mask]), float(np.max((np.abs(a - b) / np.maximum(bound, 1e-300))[mask]))
    assert np.all(a[~mask] <= FLOOR)
    return float(n.max())


def test_noalloc_matches_allocating_trace_twice(api):
    from paper_2504_21719_b300 import _lib as L
    lib = L.load()
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 10                                     # 1e6 rays of the 1e7-ray lattice
    gs = api.Scene.from_obj(sc)
    prm = api.params_from(p)
    arr = (L.rm_tx * 1)(api.tx_from(tx))
    ref = api.trace(gs, [tx], prm, record=True)
    cnt = _deposit_counts(ref["record"], [tx], p.max_depth, p.ny, p.nx)
    out = torch.empty_like(ref["maps"])
    for _ in range(2):
        out.fill_(-1.0)                                    # the call must overwrite every cell
        rc, st = _call(L, lib, gs, arr, 1, prm, out)
        assert rc == L.RM_OK, lib.rm_last_error()
        torch.cuda.synchronize()
        _same(out, ref["maps"], cnt)
        assert st.rays == ref["stats"]["rays"] and st.segments == ref["stats"]["segments"]
        assert st.deposits == ref["stats"]["deposits"]
    gs.free()


def test_noalloc_full_manhattan_map(api):
    """The whole 1e7-ray Manhattan map, where cells near the transmitter take
    the most deposits (FP32 accumulation error grows with the count)."""
    from paper_2504_21719_b300 import _lib as L
    lib = L.load()
    sc, txs, p = S.workload(2)
    tx = txs[0]
    gs = api.Scene.from_obj(sc)
    prm = api.params_from(p)
    arr = (L.rm_tx * 1)(api.tx_from(tx))
    ref = api.trace(gs, [tx], prm, record=True)
    cnt = _deposit_counts(ref["record"], [tx], p.max_depth, p.ny, p.nx)
    del ref["record"]
    out = torch.empty_like(ref["maps"])
    for _ in range(2):
        rc, st = _call(L, lib, gs, arr, 1, prm, out)
        assert rc == L.RM_OK, lib.rm_last_error()
        torch.cuda.synchronize()
        nmax = _same(out, ref["maps"], cnt)
        assert st.segments == ref["stats"]["segments"]
    assert nmax > 1000                                      # the test reaches heavily hit cells
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
    ref = api.trace(gs, txs, prm, record=True)
    cnt = _deposit_counts(ref["record"], txs, p.max_depth, p.ny, p.nx)
    out = torch.empty_like(ref["maps"])
    for _ in range(2):
        rc, st = _call(L, lib, gs, arr, len(txs), prm, out)
        assert rc == L.RM_OK, lib.rm_last_error()
        torch.cuda.synchronize()
        _same(out, ref["maps"], cnt)
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
    ref = api.trace(gs, [tx], prm, record=True)
    cnt = _deposit_counts(ref["record"], [tx], p.max_depth, p.ny, p.nx)
    out = torch.empty_like(ref["maps"])
    rc, st = _call(L, lib, gs, arr, ntx, prm, out)
    assert rc == L.RM_OK, lib.rm_last_error()
    torch.cuda.synchronize()
    _same(out, ref["maps"], cnt)
    rng = np.random.default_rng(4)
    tx.ant_pos = rng.uniform(-0.05, 0.05, size=(600, 3))
    tx.precoding = np.ones(600) / np.sqrt(600.0)
    arr2, _ = api._tx_array([tx])
    rc, _ = _call(L, lib, gs, arr2, 1, prm, out)
    assert rc == L.RM_EINVAL and b"noalloc" in lib.rm_last_error()
    gs.free()


def test_noalloc_makes_no_allocation(api):
    """Called from a thread that has never traced (so none of the library's
    per-thread buffers exist there yet), on a new stream, the entry point
    makes no allocation call; the allocating trace, in the same kind of
    thread, does.  A capturing stream is refused before anything is
    enqueued."""
    from paper_2504_21719_b300 import _lib as L
    lib = L.load()
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 100
    gs = api.Scene.from_obj(sc)
    prm = api.params_from(p)
    arr = (L.rm_tx * 1)(api.tx_from(tx))
    out = torch.empty((1, p.ny, p.nx), dtype=torch.float32, device="cuda")
    _call(L, lib, gs, arr, 1, prm, out)                    # device set-up done once
    torch.cuda.synchronize()
    res = {}

    def worker(kind):
        torch.cuda.set_device(0)
        s = torch.cuda.Stream()
        before = lib.rm_debug_alloc_count()
        if kind == "noalloc":
            rc = [_call(L, lib, gs, arr, 1, prm, out, stream=s)[0] for _ in range(2)]
        else:
            with torch.cuda.stream(s):
                api.trace(gs, [tx], prm, out=out)
            rc = [L.RM_OK]
        s.synchronize()
        res[kind] = (rc, lib.rm_debug_alloc_count() - before)

    for kind in ("noalloc", "trace"):
        t = threading.Thread(target=worker, args=(kind,))
        t.start()
        t.join()
    assert res["noalloc"][0] == [L.RM_OK, L.RM_OK], lib.rm_last_error()
    assert res["noalloc"][1] == 0, res
    assert res["trace"][1] > 0, res                       # the counter sees the allocating path
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc, _ = _call(L, lib, gs, arr, 1, prm, out, stream=s)
    assert rc == L.RM_ESTATE and b"capturing" in lib.rm_last_error()
    del g
    gs.free()
