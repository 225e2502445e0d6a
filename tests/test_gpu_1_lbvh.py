"""GPU trees == oracle trees, bit for bit (keys, order, children and child
boxes as raw FP32 bits), for both builders: the Karras LBVH and the
binned-SAH tree over the same leaves."""
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


def _compare(orc, api, sc, builder="lbvh"):
    ref = orc.lbvh(sc) if builder == "lbvh" else orc.sah_bvh(sc)
    gs = api.Scene.from_obj(sc, builder=builder)
    assert gs.info()["builder"] == builder or sc.nt == 0
    got = gs.export_bvh()
    assert np.array_equal(got["keys"], ref["keys"])
    assert np.array_equal(got["order"], ref["order"])
    assert got["nlarge"] == ref["nlarge"]
    assert np.array_equal(got["child"], ref["child"])
    assert np.array_equal(got["child_aabb"].view(np.uint32), ref["child_aabb"].view(np.uint32))
    gs.free()


@pytest.mark.parametrize("builder", ["lbvh", "sah"])
@pytest.mark.parametrize("name", list(SCENES))
def test_tree_bit_exact(orc, api, name, builder):
    _compare(orc, api, SCENES[name](), builder)


@pytest.mark.parametrize("builder", ["lbvh", "sah"])
def test_tree_bit_exact_million_triangle_city(orc, api, builder):
    _compare(orc, api, S.procedural_city(5), builder)


def test_sah_tree_bit_exact_deep_and_degenerate(orc, api):
    """Nested growing triangles reach the SAH's depth cap (middle splits below
    it); a soup with many coincident centroids takes middle splits too."""
    n = 42
    s8 = [np.float32(8.0 ** i) for i in range(n)]
    v = np.array([p for x in s8 for p in ((0, 0, 0), (x, 0, 0), (0, x, x))], np.float32)
    nested = S.Scene("nested", v, np.arange(3 * n, dtype=np.int32).reshape(n, 3), np.zeros(n, np.int32),
                     np.array([S.GROUND], np.float32))
    _compare(orc, api, nested, "sah")
    rng = np.random.default_rng(11)
    c = rng.integers(0, 5, (3000, 3)).astype(np.float32) * 10     # 125 distinct centroids
    vv = np.concatenate([c, c + [1, 0, 0], c + [0, 1, 0]]).astype(np.float32)
    tt = np.stack([np.arange(3000), np.arange(3000) + 3000, np.arange(3000) + 6000], 1).astype(np.int32)
    _compare(orc, api, S.Scene("coincident", vv, tt, np.zeros(3000, np.int32), np.array([S.GROUND], np.float32)),
             "sah")


def test_builder_argument_is_checked(api):
    """An unknown builder is RM_EINVAL before any device work; the scene can
    still be built afterwards, and a second build is RM_ESTATE."""
    import ctypes as C
    from paper_2504_21719_b300 import _lib as L
    gs = api.Scene.from_obj(S.manhattan(2, 3), build=False)
    lib = L.load()
    assert lib.rm_bvh_build_ex(gs.handle, 7, None) == L.RM_EINVAL
    assert b"builder" in lib.rm_last_error()
    assert gs.info()["builder"] is None
    assert lib.rm_bvh_build_ex(gs.handle, 2, None) == L.RM_OK
    assert gs.info()["builder"] == "sah"
    assert lib.rm_bvh_build_ex(gs.handle, 1, None) == L.RM_ESTATE
    gs.free()


def test_auto_builder(api):
    """RM_BVH_AUTO: the SAH tree above 2048 triangles, the one-block LBVH below."""
    small = api.Scene.from_obj(S.manhattan(2, 3))
    big = api.Scene.from_obj(S.procedural_city(5, ncells=30))
    assert small.info()["builder"] == "lbvh" and big.info()["builder"] == "sah"
    small.free()
    big.free()


def test_sah_and_lbvh_trace_the_same_paths(api):
    """The two trees hold the same triangles, so a trace takes the same closest
    hits through either, except where two triangles are hit at exactly the same
    distance (the first one found wins): nearly every ray's record is equal."""
    import torch
    sc, txs, p = S.workload(5)
    tx = txs[5]
    tx.ray_stride, tx.ray_begin = 997, 3
    recs, maps = [], []
    for b in ("lbvh", "sah"):
        gs = api.Scene.from_obj(sc, builder=b)
        r = api.trace(gs, [tx], p, record=True)
        recs.append(r["record"].view(tx.count(), p.max_depth + 1, 4).cpu().numpy())
        maps.append(r["maps"][0])
        gs.free()
    same = (recs[0] == recs[1]).all(axis=(1, 2))
    assert tx.count() > 90_000
    assert same.mean() > 0.999, same.mean()
    # the maps then differ only by the few differing rays' deposits
    m0, m1 = maps
    big = m0 > 1e-15
    assert torch.quantile((m1[big] - m0[big]).abs() / m0[big], 0.99) < 1e-3


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
