"""GPU cluster tree and block tree (Algorithms 1-2, Eq. 28) against the
oracle: bit-exact permutation, cluster ranges, bounding boxes and block
partition with admissibility flags."""
import os

import numpy as np
import pytest

import cavities as cv
from gpu_common import gpu_blocks, oracle_trees, rad

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

CASES = [
    ("cube768", cv.unit_cube(8), 32, 1.0),
    ("cylinder", cv.closed_cylinder(1.0, 4.0, 40, 24, 4), 16, 1.0),
    ("icosphere3", cv.icosphere(3), 20, 0.8),
    ("line37", cv.line_facets(37), 1, 1.0),
    ("plates", cv.parallel_plates(1.0, 10, 1.0), 7, 2.0),
    ("root_is_leaf", cv.unit_cube(3), 1000, 1.0),
    ("box_ragged", cv.box(1.0, 2.7, 5.3, 3, 7, 13), 5, 1.3),
]


@pytest.mark.parametrize("name,verts,leaf,eta", CASES, ids=[c[0] for c in CASES])
def test_tree_and_partition_bit_exact(name, verts, leaf, eta):
    r = rad()
    h = r.rad_build_htree(verts, leaf, eta)
    f, t, blocks = oracle_trees(verts, leaf, eta)
    tr, bl, keys = gpu_blocks(h)
    np.testing.assert_array_equal(tr["perm"], t.perm)
    nodes = t.nodes()
    pos = {id(nd): q for q, nd in enumerate(nodes)}
    assert len(nodes) == len(tr["begin"])
    for q, nd in enumerate(nodes):
        assert (tr["begin"][q], tr["end"][q], tr["level"][q]) == (nd.begin, nd.end, nd.level)
        assert tuple(tr["bbox"][q, :3]) == nd.lo and tuple(tr["bbox"][q, 3:]) == nd.hi, q
        kids = [] if nd.is_leaf else [pos[id(ch)] for ch in nd.children]
        assert list(tr["child"][q]) == (kids if kids else [-1, -1])
    assert sorted(keys) == sorted(b.key() for b in blocks)
    st = r.rad_htree_get_stats(h)
    assert st["n_blocks"] == len(blocks)
    assert st["n_admissible"] == sum(b.admissible for b in blocks)
    r.rad_htree_free(h)


def test_line_example_golden_on_gpu():
    r = rad()
    h = r.rad_build_htree(cv.line_facets(8), 1, 1.0)
    _, _, keys = gpu_blocks(h)
    want = []
    for line in open(os.path.join(GOLDEN, "line8_blocks.txt")):
        if line.startswith("#") or not line.strip():
            continue
        r0, r1, c0, c1, a = (int(x) for x in line.split())
        want.append((r0, r1, c0, c1, bool(a)))
    assert sorted(keys) == sorted(want)


def test_facet_entry_point_matches_triangle_entry_point():
    from oracle import geometry
    r = rad()
    verts = cv.closed_cylinder(1.0, 4.0, 30, 20, 3)
    f = geometry.facets_from_triangles(verts)
    h1 = r.rad_build_htree(verts, 24, 1.0)
    h2 = r.rad_build_htree_facets(f.c, f.n, f.area, 24, 1.0)
    t1, _, k1 = gpu_blocks(h1)
    t2, _, k2 = gpu_blocks(h2)
    np.testing.assert_array_equal(t1["perm"], t2["perm"])
    assert k1 == k2


def test_device_and_host_inputs_give_identical_trees():
    import torch
    r = rad()
    verts = cv.icosphere(2)
    h1 = r.rad_build_htree(verts, 12, 1.0)
    h2 = r.rad_build_htree(torch.as_tensor(verts, device="cuda"), 12, 1.0)
    assert gpu_blocks(h1)[2] == gpu_blocks(h2)[2]


def test_bad_input_is_rejected():
    r = rad()
    v = cv.unit_cube(2).copy()
    v[3, 1] = v[3, 0]          # degenerate triangle
    with pytest.raises(r.RadError) as ei:
        r.rad_build_htree(v, 4, 1.0)
    assert ei.value.code == r.RAD_EINVAL
    v = cv.unit_cube(2).copy()
    v[0, 0, 0] = np.nan
    with pytest.raises(r.RadError):
        r.rad_build_htree(v, 4, 1.0)
    with pytest.raises(r.RadError):
        r.rad_build_htree(cv.unit_cube(2), 0, 1.0)
