"""View-factor entries, Eq. (10) of the paper, §3.2.

The paper's entry is the double area integral of cos(phi_i) cos(phi_j) /
(pi R^2) over both facets (its F carries both areas, so that its reflection
matrix Eq. (11) divides by A_i).  This oracle stores the textbook view factor
F_ij = (1/A_i) * (that integral), i.e. F = diag(A)^-1 F_paper; then
Eq. (11) reads C = I - diag(1 - eps) F identically.

With the 1-point centroid rule on both facets:
  d = c_j - c_i,  r^2 = d.d,
  cos_i = n_i.d / r,  cos_j = -n_j.d / r,
  F_ij = max(cos_i, 0) max(cos_j, 0) A_j / (pi r^2)      (i != j)
  F_ii = 0   (the diagonal is zero, §3.2)
A pair that faces away on either side contributes nothing (the paper's
isolated facets have identically zero rows, §6).

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import Facets, facets_from_triangles, subdivide_triangles


def entry(fi_c, fi_n, fj_c, fj_n, A_j) -> float:
    """One F_ij by the centroid rule, written out in plain scalar Python."""
    dx = fj_c[0] - fi_c[0]
    dy = fj_c[1] - fi_c[1]
    dz = fj_c[2] - fi_c[2]
    r2 = dx * dx + dy * dy + dz * dz
    if r2 == 0.0:
        return 0.0
    r = math.sqrt(r2)
    cos_i = (fi_n[0] * dx + fi_n[1] * dy + fi_n[2] * dz) / r
    cos_j = -(fj_n[0] * dx + fj_n[1] * dy + fj_n[2] * dz) / r
    return max(cos_i, 0.0) * max(cos_j, 0.0) * A_j / (math.pi * r2)


def rows(f: Facets, row_idx, col_idx=None) -> np.ndarray:
    """Rows ``row_idx`` of F (all columns, or ``col_idx``), centroid rule."""
    ri = np.atleast_1d(np.asarray(row_idx, dtype=np.int64))
    cj = np.arange(f.size) if col_idx is None else np.atleast_1d(np.asarray(col_idx, dtype=np.int64))
    ci = f.c[ri][:, None, :]
    ni = f.n[ri][:, None, :]
    cjv = f.c[cj][None, :, :]
    njv = f.n[cj][None, :, :]
    d = cjv - ci
    r2 = np.einsum("abk,abk->ab", d, d)
    same = ri[:, None] == cj[None, :]
    r2s = np.where(r2 > 0.0, r2, 1.0)
    r = np.sqrt(r2s)
    cos_i = np.einsum("abk,abk->ab", np.broadcast_to(ni, d.shape), d) / r
    cos_j = -np.einsum("abk,abk->ab", np.broadcast_to(njv, d.shape), d) / r
    F = np.maximum(cos_i, 0.0) * np.maximum(cos_j, 0.0) * f.area[cj][None, :] / (math.pi * r2s)
    F = np.where(same | (r2 == 0.0), 0.0, F)
    return F


def dense(f: Facets, chunk: int = 512) -> np.ndarray:
    """The full N x N matrix F (FP64), assembled in row chunks."""
    N = f.size
    out = np.empty((N, N), dtype=np.float64)
    for s in range(0, N, chunk):
        out[s:s + chunk] = rows(f, np.arange(s, min(N, s + chunk)))
    return out


def dense_from_triangles(verts: np.ndarray) -> np.ndarray:
    return dense(facets_from_triangles(verts))


def composite(verts: np.ndarray, levels: int, row_idx, col_idx) -> np.ndarray:
    """F_ij by the composite centroid rule on ``4**levels`` sub-triangles.

    F_ij = (1/A_i) sum_{p in i} sum_{q in j} cos cos / (pi r^2) A_p A_q,
    the area integral of Eq. (10) divided by A_i.  Pins only.
    """
    sub = subdivide_triangles(verts, levels)          # (N, S, 3, 3)
    N, S = sub.shape[0], sub.shape[1]
    ri = np.atleast_1d(np.asarray(row_idx))
    cj = np.atleast_1d(np.asarray(col_idx))
    fi = facets_from_triangles(sub[ri].reshape(-1, 3, 3))
    fj = facets_from_triangles(sub[cj].reshape(-1, 3, 3))
    out = np.zeros((ri.size, cj.size))
    for a in range(ri.size):
        ci = fi.c[a * S:(a + 1) * S][:, None, :]
        ni = fi.n[a * S:(a + 1) * S][:, None, :]
        Ai = fi.area[a * S:(a + 1) * S]
        d = fj.c[None, :, :] - ci
        r2 = np.einsum("abk,abk->ab", d, d)
        r = np.sqrt(r2)
        cos_i = np.einsum("abk,abk->ab", np.broadcast_to(ni, d.shape), d) / r
        cos_j = -np.einsum("abk,abk->ab", np.broadcast_to(fj.n[None], d.shape), d) / r
        k = np.maximum(cos_i, 0) * np.maximum(cos_j, 0) / (math.pi * r2)
        k = k * Ai[:, None] * fj.area[None, :]                 # (S, |cj| S)
        per_j = k.sum(axis=0).reshape(cj.size, S).sum(axis=1)
        out[a] = per_j / Ai.sum()
    return out


def plate_to_plate(verts: np.ndarray, first: int, F: np.ndarray | None = None) -> float:
    """(1/A_1) sum_{i in plate 1} sum_{j in plate 2} A_i F_ij.

    Plate 1 is triangles [0, first), plate 2 the rest.  This is the view
    factor from surface 1 to surface 2 implied by the facet matrix.
    """
    f = facets_from_triangles(verts)
    if F is None:
        F = rows(f, np.arange(first))
    A1 = f.area[:first]
    return float((A1[:, None] * F[:first, first:]).sum() / A1.sum())
