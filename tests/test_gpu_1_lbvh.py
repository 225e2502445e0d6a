"""GPU LBVH == oracle LBVH, bit for bit (sorted keys, order, children and
child boxes as raw FP32 bits)."""
import numpy as np
import pytest

from synth import scenes as S

pytestmark = pytest.mark.gpu


def _dups():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    return S.Scene("dups", v, np.tile(np.array([[0, 1, 2]], np.int32), (37, 1)), np.zeros(37, np.int32),
                   np.array([S.GROUND], np.float32))


def _one():
    g = S.ground_plane()
    return S.Scene("one", g.verts, g.tris[:1], g.tri_mat[:1], g.mats)


SCENES = {
    "manhattan2": lambda: S.manhattan(2, 3),
    "manhattan4": lambda: S.manhattan(4, 7),
    "wall": S.single_wall,
    "box": S.closed_box,
    "ground": S.ground_plane,
    "city30": lambda: S.procedural_city(5, ncells=30),
    "dups": _dups,
    "one": _one,
}


def _compare(orc, api, sc):
    ref = orc.lbvh(sc)
    gs = api.Scene.from_obj(sc)
    got = gs.export_bvh()
    assert np.array_equal(got["keys"], ref["keys"])
    assert np.array_equal(got["order"], ref["order"])
    assert got["nlarge"] == ref["nlarge"]
    assert np.array_equal(got["child"], ref["child"])
    assert np.array_equal(got["child_aabb"].view(np.uint32), ref["child_aabb"].view(np.uint32))
    gs.free()


@pytest.mark.parametrize("name", list(SCENES))
def test_lbvh_bit_exact(orc, api, name):
    _compare(orc, api, SCENES[name]())


def test_lbvh_bit_exact_million_triangle_city(orc, api):
    _compare(orc, api, S.procedural_city(5))


def test_empty_scene_builds(api):
    gs = api.Scene.from_obj(S.empty_scene())
    assert gs.export_bvh()["keys"].size == 0
    gs.free()


def test_device_and_host_upload_agree(orc, api):
    """A scene uploaded from device tensors (device-side index check, synchronous)
    and from host arrays (host-side check, no wait) builds the same tree, and
    a trace from either gives the same map."""
    import torch
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 31
    gh = api.Scene.from_obj(sc)
    gd = api.Scene(torch.from_numpy(sc.verts).cuda(), torch.from_numpy(sc.tris).cuda(),
                   torch.from_numpy(sc.tri_mat).cuda(), sc.mats)
    eh, ed = gh.export_bvh(), gd.export_bvh()
    for k in ("keys", "order", "child"):
        assert np.array_equal(eh[k], ed[k]), k
    assert np.array_equal(eh["child_aabb"].view(np.uint32), ed["child_aabb"].view(np.uint32))
    mh = api.trace(gh, [tx], p)["maps"]
    md = api.trace(gd, [tx], p)["maps"]
    assert torch.equal(mh, md)
    gh.free()
    gd.free()


def test_trace_right_after_unwaited_build(orc, api):
    """Upload, build and trace back to back with no host wait in between, many
    times over (the build's large-triangle count is read by the trace): the
    maps equal those of a scene whose count was read before tracing."""
    import torch
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 97
    ref = api.Scene.from_obj(sc)
    assert ref.info()["nodes"] > 0          # waits for the build
    want = api.trace(ref, [tx], p)["maps"].clone()
    for _ in range(20):
        g = api.Scene.from_obj(sc)
        got = api.trace(g, [tx], p)["maps"]
        assert torch.equal(got, want)
        g.free()
    ref.free()


def test_scenes_built_and_traced_from_several_threads(orc, api):
    """Four host threads each upload, build (unwaited) and trace their own
    scenes on their own streams: the pinned count slots and staging buffers are
    shared or per thread, and every map equals the single-threaded one."""
    import threading

    import torch
    sc, txs, p = S.workload(2)
    tx = txs[0]
    tx.ray_stride = 211
    ref = api.Scene.from_obj(sc)
    want = api.trace(ref, [tx], p)["maps"].clone()
    ref.free()
    errors = []

    def work():
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(8):
                    g = api.Scene.from_obj(sc, stream=s)
                    got = api.trace(g, [tx], p, stream=s)["maps"]
                    s.synchronize()
                    if not torch.equal(got, want):
                        errors.append("map differs")
                    g.free()
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(repr(e))

    th = [threading.Thread(target=work) for _ in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
