"""Pins of the oracle's reference LBVH: Morton quantisation in IEEE FP32, stable
sort, and the binary radix tree's defining property checked with Python
integers on the composite keys (Karras, HPG 2012; not part of the paper,
whose implementation relies on Mitsuba's acceleration structure)."""
import numpy as np
import pytest

from synth import scenes as S


def _large_numpy(lo, hi):
    """Large triangles: largest AABB extent >= 0.25 x the scene's, unless more than 16 are."""
    ext = (hi - lo).astype(np.float32).max(1)
    es = (hi.max(0) - lo.min(0)).astype(np.float32).max()
    large = ext >= np.float32(0.25) * np.float32(es)
    if large.sum() > 16:
        large[:] = False
    return large


def _morton_numpy(scene):
    v = scene.verts.astype(np.float32)
    t = scene.tris
    p = v[t]                                   # [nt, 3, 3]
    lo, hi = p.min(1), p.max(1)
    large = _large_numpy(lo, hi)
    c2 = (lo + hi).astype(np.float32)
    small = c2[~large] if (~large).any() else c2
    cmin, cmax = small.min(0), small.max(0)
    ext = (cmax - cmin).astype(np.float32).max()      # one scale for the three axes
    scale = np.float32(2097151.0) / ext if ext > 0 else np.float32(0)
    q = ((c2 - cmin).astype(np.float32) * scale).astype(np.float32)
    qi = np.minimum(q.astype(np.uint64), np.uint64(2097151))
    keys = np.zeros(len(t), np.uint64)
    for b in range(21):
        for a, sh in ((0, 2), (1, 1), (2, 0)):
            keys |= ((qi[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + sh)
    keys[large] = np.uint64(2 ** 64 - 1)
    return keys, np.concatenate([lo, hi], 1)


def _check_tree(scene, b):
    nt = scene.nt - b["nlarge"]               # the tree covers the non-large triangles
    keys, order, child, cbox = b["keys"], b["order"], b["child"], b["child_aabb"]
    if nt <= 1:
        assert len(child) == 0
        return
    _, tbox = _morton_numpy(scene)
    comp = [(int(keys[i]) << 32) | i for i in range(nt)]  # composite key (Morton, position)
    seen = np.zeros(nt, int)
    nodes_seen = set()

    stack = [(0, 0, nt - 1)]
    while stack:
        nid, a, z = stack.pop()
        assert nid not in nodes_seen
        nodes_seen.add(nid)
        assert nid in (a, z)  # Karras: an internal node is numbered by an end of its range
        # split at the highest differing bit of the composite keys
        hb = (comp[a] ^ comp[z]).bit_length() - 1
        g = max(i for i in range(a, z) if (comp[i] >> hb) & 1 == (comp[a] >> hb) & 1)
        assert (comp[g + 1] >> hb) & 1 != (comp[a] >> hb) & 1
        L, R = child[nid]
        assert L == (~g if a == g else g) and R == (~(g + 1) if z == g + 1 else g + 1)
        for side, (c, lo_, hi_) in enumerate(((L, a, g), (R, g + 1, z))):
            want = np.concatenate([tbox[order[lo_:hi_ + 1], :3].min(0), tbox[order[lo_:hi_ + 1], 3:].max(0)])
            assert np.array_equal(cbox[nid, side].view(np.uint32), want.astype(np.float32).view(np.uint32))
            if c < 0:
                seen[~c] += 1
            else:
                stack.append((c, lo_, hi_))
    assert np.all(seen == 1) and len(nodes_seen) == nt - 1


@pytest.mark.parametrize("which", ["manhattan", "wall", "box", "city_slice"])
def test_lbvh_keys_order_tree(orc, which):
    if which == "manhattan":
        sc = S.manhattan(2, 3)
    elif which == "wall":
        sc = S.single_wall()
    elif which == "box":
        sc = S.closed_box()
    else:
        full = S.procedural_city(5, ncells=30)
        sc = full
    keys_np, _ = _morton_numpy(sc)
    keys_or, _, nl = orc.morton(sc)
    assert np.array_equal(keys_np, keys_or)
    b = orc.lbvh(sc)
    assert b["nlarge"] == nl == int((keys_or == np.uint64(2 ** 64 - 1)).sum())
    assert np.array_equal(b["order"], np.argsort(keys_or, kind="stable"))
    assert np.array_equal(b["keys"], keys_or[b["order"]])
    _check_tree(sc, b)


def test_lbvh_duplicate_keys_and_degenerate_extent(orc):
    # 37 copies of the same triangle: every key equal, extent 0 -> scale 0
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    sc = S.Scene("dups", v, np.tile(np.array([[0, 1, 2]], np.int32), (37, 1)), np.zeros(37, np.int32),
                 np.array([S.GROUND], np.float32))
    b = orc.lbvh(sc)
    # all 37 are as large as the scene, but more than 16: none is kept out of the tree
    assert b["nlarge"] == 0
    assert np.all(b["keys"] == 0) and np.array_equal(b["order"], np.arange(37))
    _check_tree(sc, b)


def test_lbvh_large_triangles_kept_out(orc):
    # the ground (1 km) of the Manhattan grid and the city (4 km) are large; buildings are not
    for sc, nl in ((S.manhattan(2, 3), 2), (S.procedural_city(5, ncells=30), 2), (S.closed_box(), 12),
                   (S.ground_and_wall(), 2)):
        b = orc.lbvh(sc)
        assert b["nlarge"] == nl
        assert sorted(b["order"][sc.nt - nl:].tolist()) == b["order"][sc.nt - nl:].tolist()
        if sc.name.startswith(("manhattan", "city")):
            assert set(b["order"][sc.nt - nl:].tolist()) == {0, 1}
        _check_tree(sc, b)


def test_lbvh_tiny(orc):
    sc = S.ground_plane()
    b = orc.lbvh(sc)
    assert b["nlarge"] == 2 and len(b["child"]) == 0 and b["order"].tolist() == [0, 1]
    wall = S.single_wall()
    b1 = orc.lbvh(S.Scene("one", wall.verts, wall.tris[:1], wall.tri_mat[:1], wall.mats))
    assert len(b1["child"]) == 0 and b1["order"].tolist() == [0]
