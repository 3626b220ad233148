"""Facet geometry of a triangle mesh (§3.1: the boundary faces of the mesh are
the facets of the cavity).

For a triangle (v0, v1, v2):
  centroid  c = ((v0 + v1) + v2) / 3
  normal    n = (v1 - v0) x (v2 - v0),  area A = |n| / 2,  unit normal n / |n|

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Facets:
    """Facet arrays, one row per facet, all float64."""
    c: np.ndarray      # (N, 3) centroids
    n: np.ndarray      # (N, 3) unit normals
    area: np.ndarray   # (N,)   areas

    @property
    def size(self) -> int:
        return int(self.area.shape[0])

    def subset(self, idx) -> "Facets":
        idx = np.asarray(idx)
        return Facets(self.c[idx], self.n[idx], self.area[idx])


def facets_from_triangles(verts: np.ndarray) -> Facets:
    """Centroid, unit normal and area of every triangle in ``verts`` (N,3,3)."""
    v = np.asarray(verts, dtype=np.float64)
    v0, v1, v2 = v[:, 0, :], v[:, 1, :], v[:, 2, :]
    c = ((v0 + v1) + v2) / 3.0
    e1 = v1 - v0
    e2 = v2 - v0
    nx = e1[:, 1] * e2[:, 2] - e1[:, 2] * e2[:, 1]
    ny = e1[:, 2] * e2[:, 0] - e1[:, 0] * e2[:, 2]
    nz = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    nn = np.sqrt(nx * nx + ny * ny + nz * nz)
    area = 0.5 * nn
    n = np.stack([nx / nn, ny / nn, nz / nn], axis=1)
    return Facets(c, n, area)


def subdivide_triangles(verts: np.ndarray, levels: int) -> np.ndarray:
    """Split every triangle into 4**levels congruent sub-triangles.

    Returns an array (N, 4**levels, 3, 3): the sub-triangles of triangle i.
    Used only by the composite-quadrature pins.
    """
    t = np.asarray(verts, dtype=np.float64)[:, None, :, :]
    for _ in range(levels):
        a, b, c = t[:, :, 0], t[:, :, 1], t[:, :, 2]
        ab, bc, ca = 0.5 * (a + b), 0.5 * (b + c), 0.5 * (c + a)
        t = np.concatenate([
            np.stack([a, ab, ca], axis=2),
            np.stack([ab, b, bc], axis=2),
            np.stack([ca, bc, c], axis=2),
            np.stack([ab, bc, ca], axis=2)], axis=1)
    return t
