"""Seeded synthetic cavity inputs shared by the tests, the oracle checks and the bench.

This module only builds triangle meshes and draws emissivities / temperatures.
It holds none of the radiation method's arithmetic (no view factors, trees,
ACA or solves), so both the CUDA path and the CPU oracle can take their inputs
from it without sharing any of the method's code.

Every mesh is returned as a float64 array ``verts`` of shape ``(N, 3, 3)``
(triangle, vertex, xyz).  Triangles are wound so that
``(v1 - v0) x (v2 - v0)`` points INTO the cavity (the facets face each other).

Workload recipe (the paper's own meshes, tetrahedral sphere clusters of its
numerical-experiments section, are not available; these synthetic cavities
stand in for them):

* ``config1``: unit cube interior, every face an 8x8 grid of squares, each
  split along its v00-v11 diagonal (768 triangles, area 1/128 each);
  emissivity U[0.3, 0.9], temperature U[300, 1200] K.
* ``config2``: closed cylinder R=1, H=4: 112 sectors x 72 rows on the side
  (16,128 triangles) and two caps of 9 rings (a 112-triangle fan in the centre
  ring, 8 quad rings) = 1,904 each; N = 19,936; emissivity U[0.3, 0.9];
  64 temperature fields U[300, 1200] K.
* ``config3``: icosphere level 6 (81,920 triangles, inward normals);
  emissivity U[0.1, 0.95]; temperature U[300, 1200] K.
* ``config4``: 256 boxes with sides (1, a, b), a, b log-uniform in [1, 8],
  target facet counts log-uniform in [2,000, 40,000].
* ``config5``: Poisson arrival stream (mean 200 req/s) of cubes, cylinders and
  spheres with 5,000-200,000 target facets.

Random numbers come from numpy's PCG64 seeded with ``20230511 + index``;
draws are made in facet order.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20230511

__all__ = [
    "Cavity", "rng_for", "grid_face", "unit_cube", "box", "closed_cylinder",
    "icosphere", "parallel_plates", "perpendicular_plates", "line_facets",
    "config1", "config2", "config3", "config4", "config5", "cylinder_for_n",
]


@dataclass
class Cavity:
    """One synthetic workload: mesh, emissivities and temperature fields."""
    name: str
    verts: np.ndarray                # (N, 3, 3) float64
    eps: np.ndarray                  # (N,) float64
    T: np.ndarray                    # (N, m) float64, Kelvin
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.verts.shape[0])


def rng_for(index: int) -> np.random.Generator:
    """PCG64 generator for workload ``index`` (seed 20230511 + index)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(index)))


def grid_face(origin, e1, e2, n1: int, n2: int) -> np.ndarray:
    """Triangulate the parallelogram ``origin + s*e1 + t*e2`` (s, t in [0,1]).

    The face is cut into ``n1 x n2`` cells; each cell (v00, v10, v01, v11) is
    split along its v00-v11 diagonal into (v00, v10, v11) and (v00, v11, v01).
    Both triangles are wound like ``e1 x e2``.
    """
    o = np.asarray(origin, dtype=np.float64)
    e1 = np.asarray(e1, dtype=np.float64)
    e2 = np.asarray(e2, dtype=np.float64)
    out = np.empty((n1 * n2 * 2, 3, 3), dtype=np.float64)
    k = 0
    for b in range(n2):
        for a in range(n1):
            s0, s1 = a / n1, (a + 1) / n1
            t0, t1 = b / n2, (b + 1) / n2
            v00 = o + s0 * e1 + t0 * e2
            v10 = o + s1 * e1 + t0 * e2
            v01 = o + s0 * e1 + t1 * e2
            v11 = o + s1 * e1 + t1 * e2
            out[k] = (v00, v10, v11)
            out[k + 1] = (v00, v11, v01)
            k += 2
    return out


def box(lx: float, ly: float, lz: float, nx: int, ny: int, nz: int) -> np.ndarray:
    """Interior of the box [0,lx]x[0,ly]x[0,lz] with inward-facing triangles.

    ``nx, ny, nz`` are the numbers of cells along each axis on every face
    that spans that axis.
    """
    X, Y, Z = float(lx), float(ly), float(lz)
    faces = [
        grid_face((0, 0, 0), (X, 0, 0), (0, Y, 0), nx, ny),   # z=0, normal +z
        grid_face((0, 0, Z), (0, Y, 0), (X, 0, 0), ny, nx),   # z=Z, normal -z
        grid_face((0, 0, 0), (0, Y, 0), (0, 0, Z), ny, nz),   # x=0, normal +x
        grid_face((X, 0, 0), (0, 0, Z), (0, Y, 0), nz, ny),   # x=X, normal -x
        grid_face((0, 0, 0), (0, 0, Z), (X, 0, 0), nz, nx),   # y=0, normal +y
        grid_face((0, Y, 0), (X, 0, 0), (0, 0, Z), nx, nz),   # y=Y, normal -y
    ]
    return np.concatenate(faces, axis=0)


def unit_cube(n: int = 8) -> np.ndarray:
    """Unit cube interior, every face an ``n x n`` grid (12 n^2 triangles)."""
    return box(1.0, 1.0, 1.0, n, n, n)


def closed_cylinder(R: float = 1.0, H: float = 4.0, n_sector: int = 112,
                    n_rows: int = 72, n_rings: int = 9) -> np.ndarray:
    """Closed cylinder interior (side + two caps), inward-facing triangles.

    Side: ``n_sector x n_rows`` quads, two triangles each.  Each cap has
    ``n_rings`` rings: a fan of ``n_sector`` triangles in the centre ring and
    two triangles per quad in the outer rings.
    """
    phi = 2.0 * np.pi * np.arange(n_sector + 1) / n_sector
    phi[-1] = 0.0
    cs, sn = np.cos(phi), np.sin(phi)
    cs[-1], sn[-1] = cs[0], sn[0]
    tris = []
    zs = H * np.arange(n_rows + 1) / n_rows
    # side: e1 along +z, e2 along +phi  =>  (e1 x e2) points to the axis
    for r in range(n_rows):
        for s in range(n_sector):
            v00 = (R * cs[s], R * sn[s], zs[r])
            v10 = (R * cs[s], R * sn[s], zs[r + 1])
            v01 = (R * cs[s + 1], R * sn[s + 1], zs[r])
            v11 = (R * cs[s + 1], R * sn[s + 1], zs[r + 1])
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    rho = R * np.arange(n_rings + 1) / n_rings
    for z, up in ((0.0, True), (H, False)):
        cap = []
        c = (0.0, 0.0, z)
        for s in range(n_sector):
            p1 = (rho[1] * cs[s], rho[1] * sn[s], z)
            p2 = (rho[1] * cs[s + 1], rho[1] * sn[s + 1], z)
            cap.append((c, p1, p2))
        for k in range(1, n_rings):
            for s in range(n_sector):
                v00 = (rho[k] * cs[s], rho[k] * sn[s], z)
                v10 = (rho[k + 1] * cs[s], rho[k + 1] * sn[s], z)
                v01 = (rho[k] * cs[s + 1], rho[k] * sn[s + 1], z)
                v11 = (rho[k + 1] * cs[s + 1], rho[k + 1] * sn[s + 1], z)
                cap.append((v00, v10, v11))
                cap.append((v00, v11, v01))
        if not up:  # top cap faces -z: swap the last two vertices
            cap = [(a, cc, b) for (a, b, cc) in cap]
        tris.extend(cap)
    return np.asarray(tris, dtype=np.float64)


_ICO_FACES = np.array([
    (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
    (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
    (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
    (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], dtype=np.int64)


def icosphere(level: int, R: float = 1.0, inward: bool = True) -> np.ndarray:
    """Icosahedron subdivided ``level`` times (20 * 4**level triangles).

    Each subdivision splits a triangle at its edge midpoints, projected to the
    sphere.  Triangles face the centre when ``inward`` is set.
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
                  (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
                  (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    tri = v[_ICO_FACES]                                   # (20, 3, 3)
    # orient every base face outward first
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    flip = np.einsum("ij,ij->i", nrm, tri.sum(axis=1)) < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]

    def unit(a):
        return a / np.linalg.norm(a, axis=-1, keepdims=True)

    for _ in range(level):
        a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
        ab, bc, ca = unit(a + b), unit(b + c), unit(c + a)
        tri = np.stack([
            np.stack([a, ab, ca], axis=1),
            np.stack([b, bc, ab], axis=1),
            np.stack([c, ca, bc], axis=1),
            np.stack([ab, bc, ca], axis=1)], axis=1).reshape(-1, 3, 3)
    tri = tri * R
    if inward:
        tri = tri[:, [0, 2, 1]]
    return np.ascontiguousarray(tri)


def parallel_plates(L: float = 1.0, n: int = 8, gap: float = 1.0) -> np.ndarray:
    """Two coaxial ``L x L`` plates at distance ``gap`` facing each other.

    Each plate is an ``n x n`` grid of squares split into two triangles.
    The first ``2 n^2`` triangles are the lower plate (normal +z).
    """
    lower = grid_face((0, 0, 0), (L, 0, 0), (0, L, 0), n, n)
    upper = grid_face((0, 0, gap), (0, L, 0), (L, 0, 0), n, n)
    return np.concatenate([lower, upper], axis=0)


def perpendicular_plates(L: float = 1.0, n: int = 8) -> np.ndarray:
    """Two ``L x L`` plates at a right angle sharing the edge x=0, z=0.

    The first ``2 n^2`` triangles lie in z=0 (normal +z), the rest in x=0
    (normal +x).
    """
    floor = grid_face((0, 0, 0), (L, 0, 0), (0, L, 0), n, n)
    wall = grid_face((0, 0, 0), (0, L, 0), (0, 0, L), n, n)
    return np.concatenate([floor, wall], axis=0)


def line_facets(n: int, spacing: float = 1.0) -> np.ndarray:
    """``n`` small triangles whose centroids lie on the x axis at ``i*spacing``.

    Each triangle is (x-d, -d, 0), (x+d, -d, 0), (x, 2d, 0) with d = spacing/8,
    so its centroid is exactly (x, 0, 0) whenever x, d are exact binary values.
    """
    d = spacing / 8.0
    out = np.empty((n, 3, 3), dtype=np.float64)
    for i in range(n):
        x = i * spacing
        out[i] = ((x - d, -d, 0.0), (x + d, -d, 0.0), (x, 2 * d, 0.0))
    return out


def _fields(rng, n: int, m: int, eps_lo: float, eps_hi: float):
    eps = rng.uniform(eps_lo, eps_hi, size=n)
    T = rng.uniform(300.0, 1200.0, size=(n, m))
    return eps, T


def config1() -> Cavity:
    """Unit cube, 8x8 squares per face, 768 triangles, FP64 workload."""
    verts = unit_cube(8)
    eps, T = _fields(rng_for(0), verts.shape[0], 1, 0.3, 0.9)
    return Cavity("unit_cube_768", verts, eps, T,
                  dict(leaf_size=32, eta_adm=1.0, aca_tol=1e-6))


def config2(m: int = 64) -> Cavity:
    """Closed cylinder R=1, H=4, 19,936 triangles, ``m`` temperature fields."""
    verts = closed_cylinder()
    eps, T = _fields(rng_for(1), verts.shape[0], m, 0.3, 0.9)
    return Cavity("closed_cylinder_19936", verts, eps, T,
                  dict(leaf_size=64, eta_adm=1.0, aca_tol=1e-5))


def config3() -> Cavity:
    """Icosphere level 6 interior, 81,920 triangles."""
    verts = icosphere(6)
    eps, T = _fields(rng_for(2), verts.shape[0], 1, 0.1, 0.95)
    return Cavity("icosphere6_81920", verts, eps, T,
                  dict(leaf_size=64, eta_adm=1.0, aca_tol=1e-7))


def _box_for_target(a: float, b: float, n_target: float) -> np.ndarray:
    sides = (1.0, a, b)
    area = 2.0 * (sides[0] * sides[1] + sides[1] * sides[2] + sides[0] * sides[2])
    h = math.sqrt(area / (n_target / 2.0))
    nx, ny, nz = (max(1, int(round(s / h))) for s in sides)
    return box(sides[0], sides[1], sides[2], nx, ny, nz)


def config4(count: int = 256, scale: float = 1.0) -> list[Cavity]:
    """``count`` boxes (1, a, b), a, b log-uniform in [1, 8], 2k-40k facets.

    ``scale`` multiplies the target facet counts (tests use a small scale).
    """
    rng = rng_for(3)
    out = []
    for c in range(count):
        a, b = np.exp(rng.uniform(0.0, math.log(8.0), size=2))
        n_target = math.exp(rng.uniform(math.log(2000.0), math.log(40000.0))) * scale
        verts = _box_for_target(float(a), float(b), max(n_target, 24.0))
        eps, T = _fields(rng, verts.shape[0], 1, 0.3, 0.9)
        out.append(Cavity(f"box_{c}", verts, eps, T,
                          dict(leaf_size=64, eta_adm=1.0, aca_tol=1e-6,
                               sides=(1.0, float(a), float(b)))))
    return out


def cylinder_for_n(n_target: float, R: float = 1.0, H: float = 4.0) -> np.ndarray:
    """Closed cylinder with roughly ``n_target`` triangles (C2 proportions)."""
    s = math.sqrt(max(n_target, 64.0) / 19936.0)
    n_sector = max(8, int(round(112 * s)))
    n_rows = max(2, int(round(72 * s)))
    n_rings = max(2, int(round(9 * s)))
    return closed_cylinder(R, H, n_sector, n_rows, n_rings)


def config5(n_requests: int = 64, rate: float = 200.0, n_lo: float = 5000.0,
            n_hi: float = 200000.0):
    """Poisson arrival stream of flux-solve requests.

    Returns a list of ``(arrival_time_s, Cavity)``; cavities are drawn
    uniformly from {cube, cylinder, sphere} with log-uniform target sizes.
    """
    rng = rng_for(4)
    t = 0.0
    out = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate)
        kind = int(rng.integers(0, 3))
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        if kind == 0:
            k = max(1, int(round(math.sqrt(n_target / 12.0))))
            verts = unit_cube(k)
        elif kind == 1:
            verts = cylinder_for_n(n_target)
        else:
            lvl = max(1, int(round(math.log(n_target / 20.0, 4.0))))
            verts = icosphere(lvl)
        eps, T = _fields(rng, verts.shape[0], 1, 0.3, 0.9)
        out.append((t, Cavity(f"req_{r}", verts, eps, T,
                              dict(leaf_size=64, eta_adm=1.0, aca_tol=1e-7))))
    return out


def config5_stream(n_cavities: int = 12, n_requests: int = 96, rate: float = 200.0, n_lo: float = 5000.0,
                   n_hi: float = 200000.0):
    """Served stream of transient-step flux solves on a pool of cavities.

    The pool holds ``n_cavities`` cavities drawn like :func:`config5`
    (cube, cylinder or sphere, log-uniform target size in [n_lo, n_hi]); each
    of the ``n_requests`` requests arrives after an exponential gap (mean
    1/rate), picks a pool cavity uniformly and carries its own emissivity and
    temperature field.  Returns ``(pool, requests)`` with ``pool`` a list of
    vertex arrays and ``requests`` a list of ``(arrival_s, cavity, eps, T)``.
    """
    rng = rng_for(5)
    pool = []
    for _ in range(n_cavities):
        kind = int(rng.integers(0, 3))
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        if kind == 0:
            verts = unit_cube(max(1, int(round(math.sqrt(n_target / 12.0)))))
        elif kind == 1:
            verts = cylinder_for_n(n_target)
        else:
            verts = icosphere(max(1, int(round(math.log(n_target / 20.0, 4.0)))))
        pool.append(verts)
    t = 0.0
    reqs = []
    for _ in range(n_requests):
        t += rng.exponential(1.0 / rate)
        c = int(rng.integers(0, n_cavities))
        eps, T = _fields(rng, pool[c].shape[0], 1, 0.3, 0.9)
        reqs.append((t, c, eps, T))
    return pool, reqs
