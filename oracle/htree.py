"""Cluster tree (Algorithm 1), admissibility (Eq. 28) and block tree
(Algorithm 2) of §4.1-4.2, written as plain recursive Python.

Readings of the paper where it leaves a choice open:

* Split (Algorithm 1 says only "a hyperplane"): the node's centroids are cut
  on the axis of largest bounding-box extent (ties: lowest axis).  The left
  child receives the floor(#tau/2) facets that come first in the order
  (coordinate on that axis, original index); the right child the rest.  Every
  node lists its facets in ascending original index, so the leaves, read left
  to right, give the permutation of §4.1 (rows and columns reordered so that
  every cluster is a contiguous range).  A node is a leaf iff #tau <= n_min.
* diam / dist of the centroid point clouds (Eq. 28): taken on axis-aligned
  bounding boxes of the centroids.  diam^2 = |hi - lo|^2,
  dist^2 = sum_k max(0, lo_t,k - hi_s,k, lo_s,k - hi_t,k)^2.  A block is
  admissible iff dist^2 > 0 and min(diam_s^2, diam_t^2) <= eta^2 dist^2
  (the squared form of Eq. 28, evaluated in FP64 left to right; the dist > 0
  guard keeps touching clusters out).
* Algorithm 2 when a cluster has no children: an inadmissible block whose row
  or column cluster is a leaf is itself a (dense) leaf block.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Cluster:
    begin: int                     # first position in tree order
    end: int                       # one past the last position
    level: int
    lo: tuple                      # bounding box of the centroids
    hi: tuple
    children: list = field(default_factory=list)

    @property
    def size(self) -> int:
        return self.end - self.begin

    @property
    def is_leaf(self) -> bool:
        return not self.children


@dataclass
class ClusterTree:
    root: Cluster
    perm: np.ndarray               # perm[p] = original facet index at position p
    n_min: int

    def nodes(self) -> list:
        """All clusters, breadth first."""
        out, frontier = [], [self.root]
        while frontier:
            out.extend(frontier)
            frontier = [ch for c in frontier for ch in c.children]
        return out

    def leaves(self) -> list:
        return [c for c in self.nodes() if c.is_leaf]


def _bbox(points: np.ndarray, idx: list):
    lo = [float(min(points[i, k] for i in idx)) for k in range(3)]
    hi = [float(max(points[i, k] for i in idx)) for k in range(3)]
    return tuple(lo), tuple(hi)


def build_cluster_tree(centroids: np.ndarray, n_min: int) -> ClusterTree:
    """T_I := BuildIndexTree(I), Algorithm 1 with the split reading above."""
    pts = np.asarray(centroids, dtype=np.float64)
    N = pts.shape[0]
    perm: list = []

    def build(tau: list, begin: int, level: int) -> Cluster:
        lo, hi = _bbox(pts, tau)
        node = Cluster(begin, begin + len(tau), level, lo, hi)
        if len(tau) <= n_min:                      # leaf index set
            perm.extend(tau)
            return node
        ext = [hi[k] - lo[k] for k in range(3)]
        axis = 0
        for k in (1, 2):
            if ext[k] > ext[axis]:
                axis = k
        order = sorted(tau, key=lambda i: (pts[i, axis] + 0.0, i))
        half = len(tau) // 2
        left = sorted(order[:half])
        right = sorted(order[half:])
        node.children = [build(left, begin, level + 1),
                         build(right, begin + half, level + 1)]
        return node

    root = build(list(range(N)), 0, 0) if N > 0 else Cluster(0, 0, 0, (0,) * 3, (0,) * 3)
    return ClusterTree(root, np.asarray(perm, dtype=np.int64), n_min)


def diam2(c: Cluster) -> float:
    dx = c.hi[0] - c.lo[0]
    dy = c.hi[1] - c.lo[1]
    dz = c.hi[2] - c.lo[2]
    return dx * dx + dy * dy + dz * dz


def dist2(s: Cluster, t: Cluster) -> float:
    g = [max(0.0, t.lo[k] - s.hi[k], s.lo[k] - t.hi[k]) for k in range(3)]
    return g[0] * g[0] + g[1] * g[1] + g[2] * g[2]


def admissible(s: Cluster, t: Cluster, eta: float) -> bool:
    """Eq. (28): min(diam A_s, diam A_t) <= eta dist(A_s, A_t), squared form."""
    d2 = dist2(s, t)
    if not d2 > 0.0:
        return False
    return min(diam2(s), diam2(t)) <= (eta * eta) * d2


@dataclass
class Block:
    row: Cluster
    col: Cluster
    admissible: bool

    def key(self):
        return (self.row.begin, self.row.end, self.col.begin, self.col.end, self.admissible)


def build_block_tree(tree: ClusterTree, eta: float) -> list:
    """T_{IxI} := BuildBlockTree(I, I), Algorithm 2; returns the leaf blocks."""
    out: list = []

    def rec(s: Cluster, t: Cluster):
        if admissible(s, t, eta):
            out.append(Block(s, t, True))
            return
        if s.is_leaf or t.is_leaf:
            out.append(Block(s, t, False))
            return
        for sc in s.children:
            for tc in t.children:
                rec(sc, tc)

    if tree.root.size > 0:
        rec(tree.root, tree.root)
    return out
