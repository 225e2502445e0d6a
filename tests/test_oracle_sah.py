"""Pins of the oracle's reference binned-SAH tree (surface-area heuristic of
MacDonald & Booth 1990 over 32 centroid bins per axis, Wald 2007; not part of
the paper, whose implementation relies on Mitsuba's acceleration structure).

The tree is checked against what its definition fixes, computed a different
way: structural invariants (leaves and node numbers are permutations, boxes
are exact unions, the large-triangle list is the LBVH's), the optimality of
every split by brute force over the candidate planes from the triangle sets
themselves (no bin accumulation, no prefix sweeps), a balanced tree in closed
form, median splits for coincident centroids, and the depth cap."""
import math

import numpy as np
import pytest

from synth import scenes as S

NB, DEPTH_CAP = 32, 32


def _tris_at(centers, size=1.0, name="pts"):
    """One small flat triangle per centre: (c - (s,0,0), c + (s,0,0), c + (0,s,0))."""
    c = np.asarray(centers, np.float32)
    s = np.float32(size)
    v = np.concatenate([c - [s, 0, 0], c + [s, 0, 0], c + [0, s, 0]]).astype(np.float32)
    n = len(c)
    tris = np.stack([np.arange(n), np.arange(n) + n, np.arange(n) + 2 * n], 1).astype(np.int32)
    return S.Scene(name, v, tris, np.zeros(n, np.int32), np.array([S.GROUND], np.float32))


def _soup(seed=3, n=600):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-100, 100, (n, 3)).astype(np.float32)
    e = rng.uniform(-2, 2, (n, 2, 3)).astype(np.float32)
    v = np.concatenate([c, c + e[:, 0], c + e[:, 1]]).astype(np.float32)
    tris = np.stack([np.arange(n), np.arange(n) + n, np.arange(n) + 2 * n], 1).astype(np.int32)
    return S.Scene("soup", v, tris, np.zeros(n, np.int32), np.array([S.GROUND], np.float32))


def _boxes(scene):
    p = scene.verts.astype(np.float32)[scene.tris]
    return np.concatenate([p.min(1), p.max(1)], 1).astype(np.float32)


def _walk(b):
    """{node id: (lo, hi, mid, depth)} from the root, checking that every
    node's leaves are one contiguous range of positions."""
    child = b["child"]
    out = {}

    def rng(c, depth):
        if c < 0:
            return ~c, ~c + 1
        lo0, hi0 = rng(child[c, 0], depth + 1)
        lo1, hi1 = rng(child[c, 1], depth + 1)
        assert hi0 == lo1, "the children's ranges must be adjacent"
        assert c not in out, "node reached twice"
        out[c] = (lo0, hi1, hi0, depth)
        return lo0, hi1

    import sys
    sys.setrecursionlimit(10000)
    if len(child):
        assert rng(0, 0) == (0, len(child) + 1)
    return out


def _half_area(box, sc):
    """dx dy + dy dz + dz dx of the box's extents scaled by sc, in FP32."""
    d = ((box[3:] - box[:3]).astype(np.float32) * np.float32(sc)).astype(np.float32)
    return np.float32(np.float32(np.float32(d[0] * d[1]) + np.float32(d[1] * d[2])) + np.float32(d[2] * d[0]))


def _scale(cl, ch):
    """2^-E with the node's largest centroid extent = f 2^E, f in [0.5, 1)."""
    _, e = math.frexp(float((ch - cl).astype(np.float32).max()))
    return np.float32(2.0 ** -e)


def _check_structure(orc, scene):
    b = orc.sah_bvh(scene)
    lb = orc.lbvh(scene)
    ns = scene.nt - b["nlarge"]
    assert b["nlarge"] == lb["nlarge"]
    # the same triangles are in the tree; the large ones end `order` as in the LBVH
    assert np.array_equal(np.sort(b["order"][:ns]), np.sort(lb["order"][:ns]))
    assert np.array_equal(b["order"][ns:], lb["order"][ns:])
    keys, _, _ = orc.morton(scene)
    assert np.array_equal(b["keys"], keys[b["order"]])
    nodes = _walk(b)
    assert sorted(nodes) == list(range(max(ns - 1, 0)))
    tb = _boxes(scene)
    for i, (lo, hi, mid, _) in nodes.items():
        assert i == (0 if (lo, hi) == (0, ns) else (mid - 1 if mid - 1 != 0 else nodes[0][2] - 1))
        for s, (a, z) in enumerate(((lo, mid), (mid, hi))):
            bx = tb[b["order"][a:z]]
            want = np.concatenate([bx[:, :3].min(0), bx[:, 3:].max(0)])
            assert np.array_equal(b["child_aabb"][i, s].view(np.uint32), want.view(np.uint32))
    return b, nodes


SCENES = {
    "manhattan": lambda: S.manhattan(2, 3),
    "soup": _soup,
    "city30": lambda: S.procedural_city(5, ncells=30),
    "wall": S.single_wall,
    "ground": S.ground_plane,
}


@pytest.mark.parametrize("name", list(SCENES))
def test_sah_tree_structure(orc, name):
    _check_structure(orc, SCENES[name]())


def _bins(c, cl, k):
    f = ((c - cl).astype(np.float32) * np.float32(k)).astype(np.float32)
    return np.minimum(f.astype(np.int64), NB - 1)


@pytest.mark.parametrize("name", ["manhattan", "soup"])
def test_every_split_is_the_best_candidate_plane(orc, name):
    """For every node: evaluate each of the 3 x 31 candidate planes from the
    triangle sets (union boxes and counts of the two sides taken directly,
    costs in FP32 on extents scaled by the node's power of two), and check
    that the tree's left child holds exactly the triangles of the first
    minimum."""
    scene = SCENES[name]()
    b, nodes = _check_structure(orc, scene)
    tb = _boxes(scene)
    c2 = (tb[:, :3] + tb[:, 3:]).astype(np.float32)
    checked = 0
    for i, (lo, hi, mid, depth) in nodes.items():
        t = b["order"][lo:hi]
        cl, ch = c2[t].min(0), c2[t].max(0)
        sc = _scale(cl, ch)
        best, pick = np.float32(np.inf), None
        for a in range(3):
            e = np.float32(ch[a] - cl[a])
            if not (e > 0) or depth >= DEPTH_CAP:
                continue
            with np.errstate(over="ignore", divide="ignore"):
                k = np.float32(np.float32(NB) / e)
            if not np.isfinite(k):
                continue
            bins = _bins(c2[t, a], cl[a], k)
            for s in range(1, NB):
                left = bins < s
                nl = int(left.sum())
                if nl == 0 or nl == len(t):
                    continue
                L, R = tb[t[left]], tb[t[~left]]
                hl = _half_area(np.concatenate([L[:, :3].min(0), L[:, 3:].max(0)]), sc)
                hr = _half_area(np.concatenate([R[:, :3].min(0), R[:, 3:].max(0)]), sc)
                cost = np.float32(np.float32(hl * np.float32(nl)) + np.float32(hr * np.float32(len(t) - nl)))
                if cost < best:
                    best, pick = cost, set(t[left].tolist())
        if pick is None:
            # no candidate: coincident centroids (the two triangles of a quad), median split
            assert depth >= DEPTH_CAP or np.array_equal(cl, ch)
            assert mid - lo == (hi - lo) // 2
        else:
            assert set(b["order"][lo:mid].tolist()) == pick, f"node {i}"
            checked += 1
    assert checked > 0.4 * len(nodes)


def test_equal_boxes_on_a_line_give_the_balanced_tree(orc):
    """64 equal flat triangles 10 m apart: the cost (10k - 8) k + (10(n-k) - 8)(n-k)
    of k boxes on the left is strictly convex and symmetric, so every node splits
    its range in half and the tree is complete with depth 6."""
    sc = _tris_at([[10.0 * i, 0.0, 0.0] for i in range(64)])
    b, nodes = _check_structure(orc, sc)
    assert b["nlarge"] == 0
    for lo, hi, mid, _ in nodes.values():
        assert mid - lo == (hi - lo) // 2
    assert max(d for *_, d in nodes.values()) == 5
    # the leaves keep the line's order (the Morton order of points on a line)
    assert np.array_equal(b["order"], np.arange(64))


def test_coincident_centroids_split_at_the_middle(orc):
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    sc = S.Scene("dups", v, np.tile(np.array([[0, 1, 2]], np.int32), (37, 1)), np.zeros(37, np.int32),
                 np.array([S.GROUND], np.float32))
    b, nodes = _check_structure(orc, sc)
    for lo, hi, mid, _ in nodes.values():
        assert mid - lo == (hi - lo) // 2
    assert np.array_equal(b["order"], orc.lbvh(sc)["order"])


def test_depth_cap_on_nested_growing_triangles(orc):
    """Triangle i spans the cube [0, 8^i]^3 (i < 42; the last is large and leaves
    the tree).  Splitting the k largest off costs s^2 ((n - k) 8^(-2k) + k) up to
    a common factor, least at k = 1 for n = 41, so without a cap the SAH peels
    one triangle off per level (depth 39).  From depth 32 on the ranges split
    at the middle, which bounds the depth by 32 + ceil(log2 n)."""
    n = 42
    s = [np.float32(8.0 ** i) for i in range(n)]
    v = np.array([p for x in s for p in ((0, 0, 0), (x, 0, 0), (0, x, x))], np.float32)
    sc = S.Scene("nested", v, np.arange(3 * n, dtype=np.int32).reshape(n, 3), np.zeros(n, np.int32),
                 np.array([S.GROUND], np.float32))
    b, nodes = _check_structure(orc, sc)
    assert b["nlarge"] == 1
    depth = max(d for *_, d in nodes.values())
    assert depth >= DEPTH_CAP                                  # the cap is reached ...
    assert depth < DEPTH_CAP + math.ceil(math.log2(n - 1))     # ... and bounds the depth
    for lo, hi, mid, d in nodes.values():
        if d < DEPTH_CAP:
            assert hi - mid == 1 and lo == 0                   # peeled: the largest goes right
        else:
            assert mid - lo == (hi - lo) // 2


def test_sah_cost_below_the_lbvh(orc):
    """The SAH tree's total internal-node area (relative to the root) is below
    the LBVH's on a city and a triangle soup."""
    def cost(bv):
        ca = bv["child_aabb"].astype(np.float64)
        internal = bv["child"] >= 0
        d = ca[..., 3:] - ca[..., :3]
        h = d[..., 0] * d[..., 1] + d[..., 1] * d[..., 2] + d[..., 2] * d[..., 0]
        root = np.concatenate([ca[0, :, :3].min(0), ca[0, :, 3:].max(0)])
        dr = root[3:] - root[:3]
        return h[internal].sum() / (dr[0] * dr[1] + dr[1] * dr[2] + dr[2] * dr[0])
    for sc in (S.procedural_city(5, ncells=30), _soup()):
        assert cost(orc.sah_bvh(sc)) < 0.95 * cost(orc.lbvh(sc))
