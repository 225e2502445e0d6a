"""Injected host-side failures on a real device: each returns its status, no
kernel faults, and the next call on the same context is correct."""
import pytest
import torch

from synth import scenes as S

pytestmark = pytest.mark.gpu


def _small():
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 101
    return sc, tx, p


def test_injected_launch_and_overflow_keep_the_context(api):
    from paper_2504_21719_b300 import _lib as L
    sc, tx, p = _small()
    gs = api.Scene.from_obj(sc)
    ref = api.trace(gs, [tx], p)["maps"].clone()
    lib = L.load()
    assert lib.rm_debug_inject(L.RM_FAULT_LAUNCH, 1) == L.RM_OK
    with pytest.raises(api.RmError, match="injected launch failure") as e:
        api.trace(gs, [tx], p)
    assert e.value.status == L.RM_ECUDA
    assert torch.equal(api.trace(gs, [tx], p)["maps"], ref)
    # an overflow report: the maps are written, the status says rays may be missing
    assert lib.rm_debug_inject(L.RM_FAULT_OVERFLOW, 1) == L.RM_OK
    out = torch.zeros_like(ref)
    with pytest.raises(api.RmError) as e:
        api.trace(gs, [tx], p, out=out)
    assert e.value.status == L.RM_EOVERFLOW
    assert torch.allclose(out, ref, rtol=2e-5, atol=0)
    # the adjoint reports the same way
    assert lib.rm_debug_inject(L.RM_FAULT_LAUNCH, 1) == L.RM_OK
    with pytest.raises(api.RmError, match="injected"):
        api.grad(gs, [tx], p, torch.ones_like(ref))
    g = api.grad(gs, [tx], p, torch.ones_like(ref))
    assert torch.isfinite(g["d_eps"]).all()
    assert torch.allclose(api.trace(gs, [tx], p)["maps"], ref, rtol=2e-5, atol=0)
    gs.free()


def test_injected_allocation_failure_then_upload(api):
    from paper_2504_21719_b300 import _lib as L
    sc, tx, p = _small()
    assert L.load().rm_debug_inject(L.RM_FAULT_ALLOC, 1) == L.RM_OK
    with pytest.raises(api.RmError) as e:
        api.Scene.from_obj(sc)
    assert e.value.status == L.RM_ENOMEM
    gs = api.Scene.from_obj(sc)
    assert float(api.trace(gs, [tx], p)["maps"].sum()) > 0.0
    gs.free()


def _deep_tree_scene():
    """377 triangles whose LBVH has a 67-level chain in which both children of
    every node are internal, and whose every box contains the point (1, 2, 3):
    each triangle spans [-2^20, q + 2^20] per axis, so its doubled centroid is
    q exactly and the Morton quantisation scale is 1; q puts one key bit per
    pair of triangles at each bit position 62..3 (the split above every pair),
    and 256 triangles share key 0 (an 8-level index-split subtree).  A ray
    from (1, 2, 3) then visits every node and, nearer child first, pushes one
    entry per level: 67 > the 64-entry traversal stack."""
    import numpy as np
    H = 2 ** 20
    qs = []
    for b in range(62, 2, -1):
        i, a = divmod(b, 3)                  # key bit 3i + 2: x, 3i + 1: y, 3i: z
        q = [0, 0, 0]
        q[2 - a] = 1 << i
        qs += [tuple(q), (q[0], q[1], q[2] + 1)]
    qs += [(0, 0, 0)] * 256 + [(2 ** 21 - 1,) * 3]
    verts, tris = [], []
    for q in qs:
        lo, hi = [-H] * 3, [c + H for c in q]
        k = len(verts)
        verts += [(lo[0], lo[1], lo[2]), (hi[0], hi[1], lo[2]), (lo[0], hi[1], hi[2])]
        tris.append((k, k + 1, k + 2))
    return S.Scene("deep-tree", np.array(verts, np.float32), np.array(tris, np.int32),
                   np.zeros(len(tris), np.int32), np.array([[3.0, 0.01, 0.2]], np.float32))


def test_traversal_stack_overflow_is_reported(orc, api):
    """A real device-side overflow: the tracer drops the 65th pending node,
    sets its status word and returns RM_EOVERFLOW (forward and adjoint); no
    trap, no wait, and the next call on the context is correct."""
    from paper_2504_21719_b300 import _lib as L
    deep = _deep_tree_scene()
    b = orc.lbvh(deep)
    depth, st, cur = 0, [], 0
    while True:                              # the tracer's order when every box is hit
        c0, c1 = b["child"][cur]
        if c0 >= 0 and c1 >= 0:
            st.append(c1)
            depth = max(depth, len(st))
            cur = c0
        elif c0 >= 0 or c1 >= 0:
            cur = max(c0, c1)
        elif st:
            cur = st.pop()
        else:
            break
    assert depth == 67 and b["nlarge"] == 0
    sc, tx, p = _small()
    gs = api.Scene.from_obj(sc)
    ref = api.trace(gs, [tx], p)["maps"].clone()
    gd = api.Scene.from_obj(deep, builder="lbvh")   # the chain is the LBVH's
    tdeep = S.Tx(pos=(1.0, 2.0, 3.0), num_rays=2000, seed=3)
    pdeep = S.TraceParams(3.5e9, 2, cell_size=1.0, nx=8, ny=8, map_origin=(0.0, 0.0, 0.0))
    with pytest.raises(api.RmError) as e:
        api.trace(gd, [tdeep], pdeep)
    assert e.value.status == L.RM_EOVERFLOW
    with pytest.raises(api.RmError) as e:
        api.grad(gd, [tdeep], pdeep, torch.ones((1, 8, 8), device="cuda"))
    assert e.value.status == L.RM_EOVERFLOW
    gd.free()
    assert torch.allclose(api.trace(gs, [tx], p)["maps"], ref, rtol=2e-5, atol=0)
    gs.free()


def test_mesh_diffraction_crossing_limit_is_reported(api):
    """The diffraction map on a mesh surface keeps at most 8 crossings per
    diffracted ray: ten stacked layers under a building's roof edges set the
    device status word (RM_EOVERFLOW, no trap); four layers do not, and the
    context stays usable."""
    import numpy as np
    from paper_2504_21719_b300 import _lib as L
    sc = S.single_box(0.0, 20.0, 0.0, 30.0, 25.0, ground=500.0)
    tx = S.Tx(pos=(-30.0, -40.0, 12.0), num_rays=1, seed=1)
    p = S.TraceParams(3.5e9, 1, cell_size=1.0, nx=8, ny=8)

    def layers(n):
        v, t = [], []
        for j in range(n):
            z = 1.0 + j
            k = len(v)
            v += [(-200.0, -200.0, z), (200.0, -200.0, z), (200.0, 200.0, z), (-200.0, 200.0, z)]
            t += [(k, k + 1, k + 2), (k, k + 2, k + 3)]
        return np.array(v, np.float32), np.array(t, np.int32)

    gs = api.Scene.from_obj(sc)
    su10 = api.surface(*layers(10))
    with pytest.raises(api.RmError) as e:
        api.diffraction_map_mesh(gs, su10, [tx], p, 256)
    assert e.value.status == L.RM_EOVERFLOW
    su10.free()
    su4 = api.surface(*layers(4))
    r = api.diffraction_map_mesh(gs, su4, [tx], p, 256)
    assert r["stats"]["deposits"] > 0
    assert float(r["maps"].sum()) > 0.0
    su4.free()
    gs.free()
