"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module generates *inputs only*: analytic surface meshes (icosphere, ellipsoid,
torus) with their exact vertex normals, incidence and observation directions, and
seeded random draws.  It performs none of the boundary-element arithmetic; the
oracle (``oracle/``) and the CUDA library each build their own RWG tables,
quadrature rules and matrices from these arrays.

The paper's own meshes (gmsh spheres by precision, the kite, the Fichera cube) are
not available, so the experiments are reproduced on analytic shapes of the same
kind and size (unit sphere with k*a of order 1..10, as in the paper's sphere study,
Section V-A, and a smooth torus).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "SurfaceMesh",
    "icosphere",
    "ellipsoid",
    "torus",
    "sphere_hierarchy",
    "torus_hierarchy",
    "hplane_directions",
    "zplane_directions",
    "fibonacci_directions",
    "monostatic_directions",
    "batched_ellipsoid_table",
]


@dataclass
class SurfaceMesh:
    """Closed triangulated surface: vertices (V x 3 float64), triangles (T x 3 int32,
    counter-clockwise seen from outside) and exact outward vertex normals (V x 3)."""

    verts: np.ndarray
    tris: np.ndarray
    vnormals: np.ndarray
    name: str = ""

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_edges(self) -> int:
        # closed, orientable, manifold triangulation: 3T = 2E
        return 3 * self.nt // 2


def _orient_outward(verts: np.ndarray, tris: np.ndarray, outward: np.ndarray) -> np.ndarray:
    """Flip triangles whose geometric normal points against the given outward direction."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, outward) < 0
    out = tris.copy()
    out[flip, 1], out[flip, 2] = tris[flip, 2], tris[flip, 1]
    return out


def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [[-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
         [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
         [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def icosphere(level: int, radius: float = 1.0) -> SurfaceMesh:
    """Icosphere with T = 20 * 4**level triangles, N = 30 * 4**level edges and
    V = 10 * 4**level + 2 vertices, all vertices on the sphere of the given radius.

    Refinement is nested: every vertex of level s is a vertex of level s+1."""
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    faces = f
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (i, j) if i < j else (j, i)
            if key in cache:
                return cache[key]
            m = (np.array(verts[i]) + np.array(verts[j])) * 0.5
            m /= np.linalg.norm(m)
            verts.append(tuple(m))
            cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        faces = np.array(nf, dtype=np.int64)
    V = np.array(verts, dtype=np.float64)
    nrm = V / np.linalg.norm(V, axis=1, keepdims=True)
    cent = V[faces].mean(axis=1)
    faces = _orient_outward(V, faces, cent)
    return SurfaceMesh(radius * nrm, faces.astype(np.int32), nrm.copy(), f"icosphere{level}")


def ellipsoid(level: int, semi_axes) -> SurfaceMesh:
    """Icosphere of the given level mapped to the ellipsoid with semi-axes (a, b, c);
    exact outward normals (x/a^2, y/b^2, z/c^2) normalised."""
    s = icosphere(level)
    ax = np.asarray(semi_axes, dtype=np.float64).reshape(1, 3)
    V = s.verts * ax
    n = V / ax**2
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    tris = _orient_outward(V, s.tris.astype(np.int64), V[s.tris].mean(axis=1) / ax**2)
    return SurfaceMesh(V, tris.astype(np.int32), n, f"ellipsoid{level}")


def torus(nu: int, nv: int, R: float = 1.0, r: float = 0.35) -> SurfaceMesh:
    """Torus (x, y, z) = ((R + r cos v) cos u, (R + r cos v) sin u, r sin v) on a
    nu x nv grid of quads, each split into two triangles: T = 2 nu nv, N = 3 nu nv,
    V = nu nv.  Doubling (nu, nv) gives a nested hierarchy."""
    iu, iv = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    u = 2 * np.pi * iu.ravel() / nu
    v = 2 * np.pi * iv.ravel() / nv
    V = np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], axis=1)
    n = np.stack([np.cos(v) * np.cos(u), np.cos(v) * np.sin(u), np.sin(v)], axis=1)

    def idx(i, j):
        return (i % nu) * nv + (j % nv)

    tris = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tris += [[a, b, c], [a, c, d]]
    tris = np.array(tris, dtype=np.int64)
    cent_n = n[tris].mean(axis=1)
    tris = _orient_outward(V, tris, cent_n)
    return SurfaceMesh(V, tris.astype(np.int32), n, f"torus{nu}x{nv}")


def sphere_hierarchy(levels, radius: float = 1.0):
    """Nested icospheres: hierarchy level l has T_l = 80 * 4**l triangles (icosphere
    refinement l + 1), so l = 0..4 spans 80 .. 20480 triangles (120 .. 30720 edges)."""
    return [icosphere(l + 1, radius) for l in levels]


def torus_hierarchy(levels, R: float = 1.0, r: float = 0.35):
    """Nested tori: hierarchy level l >= 1 is the (10 * 2**(l-1)) x (4 * 2**(l-1)) grid,
    T_l = 80 * 4**(l-1) (so levels 1..5 span 80 .. 20480 triangles)."""
    return [torus(10 * 2 ** (l - 1), 4 * 2 ** (l - 1), R, r) for l in levels]


def hplane_directions(n: int = 181) -> np.ndarray:
    """Observation directions (0, sin t, cos t), t = i * 180/(n-1) degrees: the plane
    containing the incidence direction +z and orthogonal to the x polarisation."""
    t = np.deg2rad(np.linspace(0.0, 180.0, n))
    return np.stack([np.zeros_like(t), np.sin(t), np.cos(t)], axis=1)


def zplane_directions(n: int = 361) -> np.ndarray:
    """Observation directions in the z = 0 plane, theta_i = i * 2 pi/(n - 1),
    i = 0..n-1 (the endpoint repeats theta = 0)."""
    t = np.linspace(0.0, 2 * np.pi, n)
    return np.stack([np.cos(t), np.sin(t), np.zeros_like(t)], axis=1)


def fibonacci_directions(n: int) -> np.ndarray:
    """n unit vectors on a Fibonacci sphere: z_j = 1 - (2j+1)/n, phi_j = j pi (3 - sqrt 5)."""
    j = np.arange(n, dtype=np.float64)
    z = 1.0 - (2 * j + 1) / n
    phi = j * np.pi * (3.0 - math.sqrt(5.0))
    rho = np.sqrt(1 - z * z)
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def polarisation_for(d: np.ndarray) -> np.ndarray:
    """Unit polarisation orthogonal to d: normalize(d x e_z), or e_x when d is parallel to e_z."""
    d = np.atleast_2d(d)
    p = np.cross(d, np.array([0.0, 0.0, 1.0]))
    nrm = np.linalg.norm(p, axis=1)
    p[nrm < 1e-12] = [1.0, 0.0, 0.0]
    nrm[nrm < 1e-12] = 1.0
    return p / nrm[:, None]


def monostatic_directions(n: int = 8):
    """Monostatic set: observation x_i = (sin t_i, 0, cos t_i), t_i = 45 deg * i, the
    incident wave travels along d_i = -x_i with polarisation e_y."""
    t = np.deg2rad(45.0 * np.arange(n))
    xh = np.stack([np.sin(t), np.zeros_like(t), np.cos(t)], axis=1)
    return -xh, np.tile([0.0, 1.0, 0.0], (n, 1)), xh


def batched_ellipsoid_table(n: int = 64, seed: int = 230801457):
    """Per-scatterer draws for the batched workload (numpy PCG64, seed + index):
    semi-axes U[0.5, 1.5]^3, wavenumber U[1, 6], icosphere level in {2, 3, 4}."""
    rows = []
    for i in range(n):
        g = np.random.Generator(np.random.PCG64(seed + i))
        ax = g.uniform(0.5, 1.5, size=3)
        k = g.uniform(1.0, 6.0)
        lvl = int(g.integers(2, 5))
        rows.append((ax, k, lvl))
    return rows


def gaussian_field_samples(n_samples: int, n_points: int, seed: int) -> np.ndarray:
    """Standard normal draws (n_samples x n_points), float64, PCG64(seed)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.standard_normal((n_samples, n_points))
