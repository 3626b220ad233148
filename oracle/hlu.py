"""Hierarchical block LU of the reflection matrix (§5.1) and its forward and
backward substitution (§5.2).

C = I - Lambda F (Eq. 11) is held in the block structure of F (Algorithm 2):
a cluster pair is either a leaf block of the block tree (dense, or low rank
U V^T for an admissible pair) or splits into the four pairs of its
children.  The identity only touches the dense diagonal leaves, and Lambda
scales the rows of every block (§5 opening paragraphs).

The factorisation C ~ L U (§5.1) recurses on the diagonal cluster pairs.
A diagonal pair that is a leaf gets a dense LU.  A diagonal pair with
children tau1, tau2 is treated as a 2 x 2 block matrix: its upper-left
diagonal block is factorised first (recursively); the off-diagonal blocks
then become the off-diagonal factors by one triangular solve each (the
upper-right block against the unit lower factor of the upper-left block,
the lower-left block against its upper factor from the right); finally the
lower-right block is replaced by its Schur complement (the lower-left
factor times the upper-right factor subtracted from it) and factorised
recursively.  Every block produced this way is brought back into the block
format of its pair, the ranks of its low-rank leaves truncated at the
relative accuracy eps_rel by the singular-value decay (§5.1).  This
oracle forms those products and substitutions exactly (as dense arrays)
and then truncates them leaf by leaf, which is the defined result of
"product, then truncation into the block format"; it is slow and meant
for small N.  The dense leaf LU has no pivoting (C is strictly diagonally
dominant by rows whenever max(1 - eps_i) * max_i sum_j F_ij < 1, which
holds for the cavities of the tests).  L is unit lower triangular; L and
U are stored together, LAPACK style, in the same block structure.

The solve x = U^-1 (L^-1 b) (§5.2) is the plain forward and backward
substitution with those factors; like the product it adds no approximation.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import solve_triangular

from .htree import build_block_tree, build_cluster_tree


@dataclass
class HNode:
    """Block of the pair (rows r0:r1, columns c0:c1) in tree order."""
    r0: int
    r1: int
    c0: int
    c1: int
    D: np.ndarray | None = None          # dense leaf
    U: np.ndarray | None = None          # low-rank leaf U V^T
    V: np.ndarray | None = None
    children: list = field(default_factory=list)   # [[A11, A12], [A21, A22]]

    @property
    def is_leaf(self) -> bool:
        return not self.children

    @property
    def low_rank(self) -> bool:
        return self.U is not None


def _structure(tree, eta: float):
    """Block structure of Algorithm 2 as nested cluster pairs."""
    leaves = {(b.row.begin, b.row.end, b.col.begin, b.col.end): b.admissible for b in build_block_tree(tree, eta)}

    def rec(s, t):
        key = (s.begin, s.end, t.begin, t.end)
        if key in leaves:
            node = HNode(*key)
            node.U = np.zeros((s.size, 0)) if leaves[key] else None
            return node
        node = HNode(*key)
        node.children = [[rec(s.children[0], t.children[0]), rec(s.children[0], t.children[1])],
                         [rec(s.children[1], t.children[0]), rec(s.children[1], t.children[1])]]
        return node

    return rec(tree.root, tree.root)


def truncate_dense(M: np.ndarray, tol: float):
    """U V^T = the best approximation of M of the smallest rank r with
    sqrt(sum_{i >= r} s_i^2) <= tol ||M||_F (singular-value decay)."""
    if M.size == 0:
        return np.zeros((M.shape[0], 0)), np.zeros((M.shape[1], 0))
    W, s, Zt = np.linalg.svd(M, full_matrices=False)
    total = float((s * s).sum())
    if total == 0.0:
        return np.zeros((M.shape[0], 0)), np.zeros((M.shape[1], 0))
    tail = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])
    r = next(r for r in range(0, s.size + 1) if tail[r] <= tol * tol * total)
    return W[:, :r] * s[:r], Zt[:r].T


def to_dense(node: HNode) -> np.ndarray:
    if node.is_leaf:
        if node.low_rank:
            return node.U @ node.V.T
        return node.D.copy()
    return np.block([[to_dense(node.children[0][0]), to_dense(node.children[0][1])],
                     [to_dense(node.children[1][0]), to_dense(node.children[1][1])]])


def fill(node: HNode, M: np.ndarray, tol: float) -> None:
    """Store the block M (the pair's full extent) in node's format: dense
    leaves take their entries, low-rank leaves their truncation at tol."""
    if node.is_leaf:
        if node.low_rank:
            node.U, node.V = truncate_dense(M, tol)
        else:
            node.D = M.copy()
        return
    m1 = node.children[0][0].r1 - node.r0
    n1 = node.children[0][0].c1 - node.c0
    fill(node.children[0][0], M[:m1, :n1], tol)
    fill(node.children[0][1], M[:m1, n1:], tol)
    fill(node.children[1][0], M[m1:, :n1], tol)
    fill(node.children[1][1], M[m1:, n1:], tol)


def _lower_unit(LU: np.ndarray) -> np.ndarray:
    return np.tril(LU, -1) + np.eye(LU.shape[0])


def _dense_lu_nopivot(A: np.ndarray) -> np.ndarray:
    """Doolittle LU without pivoting, L (unit, below) and U (on and above)
    stored together."""
    A = A.copy()
    n = A.shape[0]
    for k in range(n):
        if A[k, k] == 0.0:
            raise ZeroDivisionError("zero pivot")
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A


def hlu(node: HNode, tol: float) -> None:
    """Block LU of a diagonal pair (§5.1), in place: node ends up holding
    L and U together."""
    if node.is_leaf:
        node.D = _dense_lu_nopivot(node.D)
        return
    (A11, A12), (A21, A22) = node.children
    hlu(A11, tol)
    LU11 = to_dense(A11)
    L11, U11 = _lower_unit(LU11), np.triu(LU11)
    # off-diagonal factors: L11 U12 = C12 and L21 U11 = C21
    fill(A12, solve_triangular(L11, to_dense(A12), lower=True, unit_diagonal=True), tol)
    fill(A21, solve_triangular(U11.T, to_dense(A21).T, lower=True).T, tol)
    # Schur complement of the upper-left block
    fill(A22, to_dense(A22) - to_dense(A21) @ to_dense(A12), tol)
    hlu(A22, tol)


def matvec(node: HNode, x: np.ndarray) -> np.ndarray:
    """Block times vector following the block structure: U (V^T x) in a
    low-rank leaf, D x in a dense one."""
    if node.is_leaf:
        return node.U @ (node.V.T @ x) if node.low_rank else node.D @ x
    n1 = node.children[0][0].c1 - node.c0
    top = matvec(node.children[0][0], x[:n1]) + matvec(node.children[0][1], x[n1:])
    bot = matvec(node.children[1][0], x[:n1]) + matvec(node.children[1][1], x[n1:])
    return np.concatenate([top, bot])


def forward(node: HNode, b: np.ndarray) -> np.ndarray:
    """L y = b on a factored diagonal pair (unit lower L): y1 from L11,
    then L22 y2 = b2 - L21 y1 (§5.2, recursively)."""
    if node.is_leaf:
        return solve_triangular(_lower_unit(node.D), b, lower=True, unit_diagonal=True)
    m1 = node.children[0][0].r1 - node.r0
    y1 = forward(node.children[0][0], b[:m1])
    y2 = forward(node.children[1][1], b[m1:] - matvec(node.children[1][0], y1))
    return np.concatenate([y1, y2])


def backward(node: HNode, y: np.ndarray) -> np.ndarray:
    """U x = y on a factored diagonal pair: x2 from U22, then
    U11 x1 = y1 - U12 x2 (§5.2, recursively)."""
    if node.is_leaf:
        return solve_triangular(np.triu(node.D), y, lower=False)
    m1 = node.children[0][0].r1 - node.r0
    x2 = backward(node.children[1][1], y[m1:])
    x1 = backward(node.children[0][0], y[:m1] - matvec(node.children[0][1], x2))
    return np.concatenate([x1, x2])


@dataclass
class HLU:
    """L U ~ C in tree order (perm: tree position -> facet)."""
    N: int
    perm: np.ndarray
    root: HNode

    def factors(self):
        LU = to_dense(self.root)
        return _lower_unit(LU), np.triu(LU)

    def solve(self, b: np.ndarray) -> np.ndarray:
        """x = U^-1 (L^-1 b) (§5.2), b and x in facet order."""
        L, U = self.factors()
        bt = np.asarray(b, dtype=np.float64)[self.perm]
        y = solve_triangular(L, bt, lower=True, unit_diagonal=True)
        xt = solve_triangular(U, y, lower=False)
        x = np.empty_like(xt)
        x[self.perm] = xt
        return x

    def solve_blocks(self, b: np.ndarray) -> np.ndarray:
        """The same solve through the block structure: forward and backward
        substitution by pairs, low-rank blocks applied as U (V^T x)."""
        bt = np.asarray(b, dtype=np.float64)[self.perm]
        xt = backward(self.root, forward(self.root, bt))
        x = np.empty_like(xt)
        x[self.perm] = xt
        return x

    def stored_entries(self) -> int:
        """Entries kept by the factors: m n per dense leaf, k (m + n) per
        low-rank leaf."""
        def rec(nd):
            if nd.is_leaf:
                if nd.low_rank:
                    return nd.U.shape[1] * ((nd.r1 - nd.r0) + (nd.c1 - nd.c0))
                return nd.D.size
            return sum(rec(c) for row in nd.children for c in row)
        return rec(self.root)


def factor(F: np.ndarray, eps: np.ndarray, centroids: np.ndarray, n_min: int, eta: float, tol: float) -> HLU:
    """H-LU of C = I - diag(1 - eps) F (Eq. 11) in the block structure of
    F: the blocks of C are stored exactly except for the truncation of its
    admissible blocks at tol, then factorised with truncation at tol."""
    tree = build_cluster_tree(np.asarray(centroids, dtype=np.float64), n_min)
    perm = tree.perm
    C = np.eye(F.shape[0]) - (1.0 - np.asarray(eps, dtype=np.float64))[:, None] * np.asarray(F, dtype=np.float64)
    Ct = C[np.ix_(perm, perm)]
    root = _structure(tree, eta)
    fill(root, Ct, tol)
    hlu(root, tol)
    return HLU(F.shape[0], perm, root)
