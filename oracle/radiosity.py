"""Reflection system and cavity flux, §3.2 Eqs. (11)-(12): the paper's
"Direct solve" (§6.2), dense and in FP64.

With the textbook F = diag(A)^-1 F_paper (see ``viewfactor``):
  C = I - diag(1 - eps) F                                        Eq. (11)
  q_i = (sigma eps_i / A_i) sum_j eps_j sum_k F^paper_ik C^-1_kj (eta_j - eta_i)
      = sigma eps_i [ (F y)_i - eta_i (F z)_i ],                 Eq. (12)
  y = C^-1 (eps o eta),  z = C^-1 eps,  eta = T^4  (radiation power, Eq. 8).
q_i is the net flux INTO facet i (W/m^2).

The solves use numpy.linalg.solve (LAPACK dgesv, LU with partial pivoting).

Also here: sampled exact rows for cavities too large to assemble densely,
and the error bound used with them.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import numpy as np

from . import viewfactor
from .geometry import Facets


def close_cavity(F: np.ndarray):
    """Closed-cavity treatment of §6 (Eqs. rowsum, clamped_rowsum, F_closed),
    with the textbook F: s_i = sum_j F_ij (the paper's (1/A_i) sum_j of its
    area-weighted entries), c_i = s_i clamped to [0, 1], and every row with
    c_i != 0 divided by c_i.  Returns (F_closed, s, c)."""
    F = np.asarray(F, dtype=np.float64)
    s = F.sum(axis=1)
    c = np.clip(s, 0.0, 1.0)
    scale = np.where(c != 0.0, 1.0 / np.where(c != 0.0, c, 1.0), 1.0)
    return F * scale[:, None], s, c


def reflection_matrix(F: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """C = I - diag(1 - eps) F, Eq. (11)."""
    N = F.shape[0]
    return np.eye(N) - (1.0 - np.asarray(eps))[:, None] * F


def solve_flux(F: np.ndarray, eps: np.ndarray, T: np.ndarray, sigma: float):
    """Direct solve of Eq. (11) and the facet flux Eq. (12).

    ``T`` is (N,) or (N, m).  Returns (q, Y, z) with q shaped like T.
    """
    eps = np.asarray(eps, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    one = T.ndim == 1
    T2 = T[:, None] if one else T
    eta = T2 ** 4
    B = np.concatenate([eps[:, None] * eta, eps[:, None]], axis=1)
    C = reflection_matrix(F, eps)
    sol = np.linalg.solve(C, B)
    Y, z = sol[:, :-1], sol[:, -1]
    FY = F @ Y
    Fz = F @ z
    q = sigma * eps[:, None] * (FY - eta * Fz[:, None])
    return (q[:, 0] if one else q), Y, z


def two_planes_flux(eps1, eps2, T1, T2, sigma):
    """Eq. (5): net flux between two infinite grey planes (from 1 to 2)."""
    return sigma * eps1 * eps2 * (T1 ** 4 - T2 ** 4) / (1.0 - (1.0 - eps1) * (1.0 - eps2))


def matvec_rows(f: Facets, row_idx, x: np.ndarray, chunk: int = 64) -> np.ndarray:
    """(F x)_i for the sampled rows, entries evaluated exactly on the fly."""
    ri = np.asarray(row_idx)
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((ri.size,) + x.shape[1:])
    for s in range(0, ri.size, chunk):
        Fr = viewfactor.rows(f, ri[s:s + chunk])
        out[s:s + chunk] = Fr @ x
    return out


def residual_rows(f: Facets, eps: np.ndarray, row_idx, y: np.ndarray, b: np.ndarray):
    """r_i = b_i - (y_i - (1 - eps_i)(F y)_i) on the sampled rows, Eq. (11)."""
    ri = np.asarray(row_idx)
    Fy = matvec_rows(f, ri, y)
    e = np.asarray(eps)[ri]
    if y.ndim > 1:
        e = e[:, None]
    return b[ri] - (y[ri] - (1.0 - e) * Fy)


def rowsum_rows(f: Facets, row_idx) -> np.ndarray:
    """Exact row sums sum_j F_ij (the scaled row sum s_i of Eq. 32)."""
    ri = np.asarray(row_idx)
    return np.array([viewfactor.rows(f, [i]).sum() for i in ri])
