"""Adaptive cross approximation of an admissible block, §4.3.

The method builds row and column pivot sets R, C and the cross
X ~ X(:,C) X(R,C)^-1 X(R,:)  (Eq. 30), written as rank-one terms
X ~ U V^T = sum_k u_k v_k^T, until the block satisfies
||X - U V^T|| / ||X|| <= eps_rel  (Eq. 31; Frobenius norm, which is the norm
of the paper's Table 2, §6.3).

Two pivoting rules (§1: the paper uses full pivoting and names partial
pivoting as the faster, less reliable alternative):

* ``full``: the residual R_k = X - sum_{l<=k} u_l v_l^T is kept whole; the
  pivot is the entry of largest modulus (ties: lowest (row, column) in
  row-major order); u = R(:, j*), v = R(i*, :) / R(i*, j*).  It stops as soon
  as ||R_k||_F <= eps_rel ||X||_F, which is Eq. (31) exactly.
* ``partial``: only rows and columns are evaluated.  First pivot row: local
  row 0.  Column pivot: argmax |residual row| (ties: lowest).  A residual row
  whose largest modulus is <= max(1e-300, 1e-14 * largest pivot so far) is
  marked used and the lowest unused row is tried instead.  Next row: argmax
  |u_k| over unused rows.  Stop when |u_k| |v_k| <= eps_rel ||S_k||_F, with
  ||S_k||_F^2 = ||S_{k-1}||_F^2 + 2 sum_{l<k} (u_k.u_l)(v_k.v_l)
  + |u_k|^2 |v_k|^2, the Frobenius norm of the current cross.  This is the
  plain rule and nothing more: the stop is an estimate, and (as the paper
  warns) it can fire while rows the pivots never visited are still poorly
  approximated, so only full pivoting meets Eq. (31) exactly.

Both return (U, V, converged) with U (m, k), V (n, k).  ``converged`` is
False when the rank cap was reached first (the caller then stores the block
dense).

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import math

import numpy as np


def aca_full(X: np.ndarray, tol: float, max_rank: int):
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    R = X.copy()
    normX = math.sqrt(float((X * X).sum()))
    us, vs, rows, cols = [], [], [], []
    while True:
        normR = math.sqrt(float((R * R).sum()))
        if normR <= tol * normX:
            return _stack(us, m), _stack(vs, n), True, rows, cols
        if len(us) >= max_rank:
            return _stack(us, m), _stack(vs, n), False, rows, cols
        flat = int(np.argmax(np.abs(R)))
        i, j = divmod(flat, n)
        piv = R[i, j]
        u = R[:, j].copy()
        v = R[i, :] / piv
        R = R - np.outer(u, v)
        us.append(u)
        vs.append(v)
        rows.append(i)
        cols.append(j)


def aca_partial(get_row, get_col, m: int, n: int, tol: float, max_rank: int,
                stats: dict | None = None):
    """``get_row(i)`` -> X[i, :] (n,), ``get_col(j)`` -> X[:, j] (m,).

    If ``stats`` is given it receives ``norm2_S`` (the running estimate of
    ||U V^T||_F^2) and ``rows`` (the pivot rows, in order).
    """
    us, vs = [], []
    used = np.zeros(m, dtype=bool)
    norm2_S = 0.0
    scale = 0.0
    i = 0
    while True:
        if len(us) >= max_rank:
            return _stack(us, m), _stack(vs, n), False
        r = np.array(get_row(i), dtype=np.float64)
        for u_l, v_l in zip(us, vs):
            r = r - u_l[i] * v_l
        used[i] = True
        j = int(np.argmax(np.abs(r)))
        if abs(r[j]) <= max(1e-300, 1e-14 * scale):
            free = np.flatnonzero(~used)
            if free.size == 0:
                return _stack(us, m), _stack(vs, n), True
            i = int(free[0])
            continue
        scale = max(scale, abs(r[j]))
        v = r / r[j]
        u = np.array(get_col(j), dtype=np.float64)
        for u_l, v_l in zip(us, vs):
            u = u - v_l[j] * u_l
        uu = float(u @ u)
        vv = float(v @ v)
        cross = 0.0
        for u_l, v_l in zip(us, vs):
            cross += float(u @ u_l) * float(v @ v_l)
        norm2_S = norm2_S + 2.0 * cross + uu * vv
        if stats is not None:
            stats["norm2_S"] = norm2_S
            stats.setdefault("rows", []).append(i)
        us.append(u)
        vs.append(v)
        if math.sqrt(uu) * math.sqrt(vv) <= tol * math.sqrt(max(norm2_S, 0.0)):
            return _stack(us, m), _stack(vs, n), True
        cand = np.where(used, -1.0, np.abs(u))
        if not (cand >= 0).any():
            return _stack(us, m), _stack(vs, n), True
        i = int(np.argmax(cand))


def truncate(U: np.ndarray, V: np.ndarray, tol: float):
    """Rank truncation of a cross U V^T (§4.3 postprocessing into standard
    form; §5.1 truncates ranks at the relative accuracy eps_rel from the
    singular-value decay): with U = Q_U R_U, V = Q_V R_V and the SVD
    R_U R_V^T = W diag(s) Z^T, keep the smallest r with
    sqrt(sum_{i >= r} s_i^2) <= tol * sqrt(sum_i s_i^2) and return
    (Q_U W_r diag(s_r), Q_V Z_r), r >= 1 unless U V^T = 0."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    k = U.shape[1]
    if k == 0:
        return U, V
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V)
    W, s, Zt = np.linalg.svd(Ru @ Rv.T)
    total = float((s * s).sum())
    if total == 0.0:
        return U[:, :0], V[:, :0]
    tail = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])   # tail[r] = sum_{i >= r} s_i^2
    r = next(r for r in range(1, k + 1) if tail[r] <= tol * tol * total)
    return Qu @ W[:, :r] * s[:r], Qv @ Zt[:r].T


def _stack(vecs, length):
    if not vecs:
        return np.zeros((length, 0))
    return np.stack(vecs, axis=1)
