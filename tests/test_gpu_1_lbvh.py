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
