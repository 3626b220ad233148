"""Hierarchical block low-rank view-factor matrix (§4, items a-c) and its
matrix-vector product (§5.2).

Build: cluster tree (Algorithm 1), block tree (Algorithm 2); inadmissible
leaf blocks are stored dense (entries by Eq. 10, centroid rule); admissible
blocks are approximated by ACA (§4.3) to eps_rel, or stored dense when ACA
hits its rank cap.  The default pivoting is full pivoting, the paper's
choice (§1), which meets Eq. (31) exactly; the plain partial-pivot rule is
available as ``pivoting="partial"``.

Matvec: y = F x is the plain sum, over the leaf blocks sigma x tau, of
D x_tau (dense) or U (V^T x_tau) (low rank), in tree order, followed by the
inverse permutation.  The paper notes this product adds no approximation
beyond the blocks themselves.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import viewfactor
from .aca import aca_full, aca_partial
from .geometry import Facets
from .htree import build_block_tree, build_cluster_tree


@dataclass
class HLeaf:
    r0: int
    r1: int
    c0: int
    c1: int
    admissible: bool
    D: np.ndarray | None = None     # dense block (m, n)
    U: np.ndarray | None = None     # (m, k)
    V: np.ndarray | None = None     # (n, k)

    @property
    def rank(self) -> int:
        return -1 if self.U is None else self.U.shape[1]


@dataclass
class HMatrix:
    N: int
    perm: np.ndarray
    leaves: list

    def matvec(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        xt = x[self.perm]
        yt = np.zeros_like(xt)
        for b in self.leaves:
            xs = xt[b.c0:b.c1]
            if b.U is not None:
                yt[b.r0:b.r1] += b.U @ (b.V.T @ xs)
            else:
                yt[b.r0:b.r1] += b.D @ xs
        y = np.empty_like(yt)
        y[self.perm] = yt
        return y

    def to_dense(self) -> np.ndarray:
        Ft = np.zeros((self.N, self.N))
        for b in self.leaves:
            Ft[b.r0:b.r1, b.c0:b.c1] = b.D if b.U is None else b.U @ b.V.T
        F = np.empty_like(Ft)
        F[np.ix_(self.perm, self.perm)] = Ft
        return F


def build(f: Facets, n_min: int, eta: float, tol: float, pivoting: str = "full",
          max_rank: int | None = None) -> HMatrix:
    tree = build_cluster_tree(f.c, n_min)
    perm = tree.perm
    ft = f.subset(perm)
    leaves = []
    for blk in build_block_tree(tree, eta):
        r0, r1, c0, c1 = blk.row.begin, blk.row.end, blk.col.begin, blk.col.end
        rows = np.arange(r0, r1)
        cols = np.arange(c0, c1)
        if not blk.admissible:
            leaves.append(HLeaf(r0, r1, c0, c1, False, D=_block(ft, rows, cols)))
            continue
        m, n = r1 - r0, c1 - c0
        cap = max_rank if max_rank is not None else max(1, min(m, n) // 2)
        if pivoting == "full":
            U, V, ok, _, _ = aca_full(_block(ft, rows, cols), tol, cap)
        else:
            U, V, ok = aca_partial(lambda i: _block(ft, [r0 + i], cols)[0],
                                   lambda j: _block(ft, rows, [c0 + j])[:, 0],
                                   m, n, tol, cap)
        if ok:
            leaves.append(HLeaf(r0, r1, c0, c1, True, U=U, V=V))
        else:
            leaves.append(HLeaf(r0, r1, c0, c1, True, D=_block(ft, rows, cols)))
    return HMatrix(f.size, perm, leaves)


def _block(ft: Facets, rows, cols) -> np.ndarray:
    # F entries between facets in tree order: the subset keeps original
    # geometry, so the diagonal test inside viewfactor.rows uses tree
    # positions, which coincide with facet identity after the permutation.
    return viewfactor.rows(ft, rows, cols)
