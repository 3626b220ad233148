"""Pins for the oracle's cluster tree (Algorithm 1) and block tree
(Algorithm 2 with the admissibility condition Eq. 28): brute-force
invariants and a hand-derived 1-D block structure."""
import os

import numpy as np
import pytest

import cavities as cv
from oracle import geometry, htree

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tree(verts, n_min):
    f = geometry.facets_from_triangles(verts)
    return f, htree.build_cluster_tree(f.c, n_min)


def test_line_example_matches_hand_derivation():
    f, t = _tree(cv.line_facets(8), 1)
    np.testing.assert_array_equal(f.c[:, 0], np.arange(8.0))
    assert (f.c[:, 1:] == 0).all()
    np.testing.assert_array_equal(t.perm, np.arange(8))
    got = sorted(b.key() for b in htree.build_block_tree(t, 1.0))
    want = []
    for line in open(os.path.join(GOLDEN, "line8_blocks.txt")):
        if line.startswith("#") or not line.strip():
            continue
        r0, r1, c0, c1, a = (int(x) for x in line.split())
        want.append((r0, r1, c0, c1, bool(a)))
    assert got == sorted(want)


@pytest.mark.parametrize("verts,n_min", [
    (cv.unit_cube(4), 7),
    (cv.closed_cylinder(1.0, 4.0, 20, 9, 3), 16),
    (cv.icosphere(2), 10),
    (cv.line_facets(37), 1),
])
def test_cluster_tree_brute_force(verts, n_min):
    f, t = _tree(verts, n_min)
    N = f.size
    assert sorted(t.perm.tolist()) == list(range(N))
    pos = np.empty(N, dtype=int)
    pos[t.perm] = np.arange(N)
    for node in t.nodes():
        members = t.perm[node.begin:node.end]
        pts = f.c[members]
        # bounding box is that of the member centroids
        assert tuple(pts.min(axis=0)) == node.lo and tuple(pts.max(axis=0)) == node.hi
        if node.is_leaf:
            assert node.size <= n_min
            # inside a leaf facets keep ascending original index
            assert (np.diff(members) > 0).all()
            continue
        assert node.size > n_min
        L, R = node.children
        assert L.begin == node.begin and L.end == R.begin and R.end == node.end
        assert L.size == node.size // 2
        ext = pts.max(axis=0) - pts.min(axis=0)
        axis = int(np.argmax(ext))          # first maximum = lowest axis on ties
        lk = [(f.c[i, axis], i) for i in t.perm[L.begin:L.end]]
        rk = [(f.c[i, axis], i) for i in t.perm[R.begin:R.end]]
        assert max(lk) < min(rk)


@pytest.mark.parametrize("verts,n_min,eta", [
    (cv.unit_cube(4), 6, 1.0),
    (cv.closed_cylinder(1.0, 4.0, 20, 9, 3), 12, 1.0),
    (cv.icosphere(2), 8, 0.7),
    (cv.parallel_plates(1.0, 6, 1.0), 9, 2.0),
])
def test_block_tree_tiles_once_and_admissible_blocks_are_separated(verts, n_min, eta):
    f, t = _tree(verts, n_min)
    N = f.size
    cover = np.zeros((N, N), dtype=np.int32)
    blocks = htree.build_block_tree(t, eta)
    n_adm = 0
    for b in blocks:
        cover[b.row.begin:b.row.end, b.col.begin:b.col.end] += 1
        ps = f.c[t.perm[b.row.begin:b.row.end]]
        pt = f.c[t.perm[b.col.begin:b.col.end]]
        if b.admissible:
            n_adm += 1
            # true diameters and distance of the point clouds, brute force
            dmin = np.sqrt(((ps[:, None, :] - pt[None, :, :]) ** 2).sum(-1)).min()
            ds = np.sqrt(((ps[:, None, :] - ps[None, :, :]) ** 2).sum(-1)).max()
            dt = np.sqrt(((pt[:, None, :] - pt[None, :, :]) ** 2).sum(-1)).max()
            assert dmin > 0
            assert min(ds, dt) <= eta * dmin * (1 + 1e-12)
        else:
            # dense leaf: either cluster is a leaf (Algorithm 2 cannot recurse)
            assert b.row.is_leaf or b.col.is_leaf
            assert not htree.admissible(b.row, b.col, eta)
    assert (cover == 1).all()
    assert n_adm > 0


def test_touching_and_identical_clusters_are_never_admissible():
    f, t = _tree(cv.unit_cube(2), 2)
    for node in t.nodes():
        assert not htree.admissible(node, node, 1e9)
