"""Helpers for the GPU parity tests (imported only by tests marked gpu)."""
import numpy as np

from oracle import geometry, htree, viewfactor


def rad():
    import paper_2305_06891_gb300 as r
    return r


def oracle_trees(verts, leaf, eta):
    f = geometry.facets_from_triangles(verts)
    t = htree.build_cluster_tree(f.c, leaf)
    return f, t, htree.build_block_tree(t, eta)


def gpu_blocks(h):
    """Export the GPU block partition as sorted tuples plus the raw arrays."""
    r = rad()
    tr = r.rad_htree_export_tree(h)
    bl = r.rad_htree_export_blocks(h)
    b, e = tr["begin"], tr["end"]
    keys = [(int(b[rn]), int(e[rn]), int(b[cn]), int(e[cn]), bool(a))
            for rn, cn, a in zip(bl["row_node"], bl["col_node"], bl["admissible"])]
    return tr, bl, keys


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dense_tree_order(verts, perm):
    f = geometry.facets_from_triangles(verts)
    F = viewfactor.dense(f)
    return F, F[np.ix_(perm, perm)]
