"""Seeded synthetic inputs: surface meshes and incident-pulse parameters.

This module is shared by the tests, the benchmark and the oracle's callers.  It
holds geometry generation and random draws only -- no quadrature, no kernel, no
transform, nothing of the boundary-element method's arithmetic.

Meshes stand in for the scatterers of Sec. 7 (the unit sphere approximated by
flat triangles, Sec. 7.1) and for the ellipsoid / rounded cube / torus shapes of
the batched and serving workloads.  All meshes are closed, made of flat
triangles with outward counter-clockwise vertex order, vertices as an (nv, 3)
float64 array and triangles as an (nt, 3) int32 array.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 20060518


@dataclass
class Mesh:
    xyz: np.ndarray   # (nv, 3) float64
    tri: np.ndarray   # (nt, 3) int32, outward CCW

    @property
    def nt(self) -> int:
        return int(self.tri.shape[0])

    @property
    def nv(self) -> int:
        return int(self.xyz.shape[0])


def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def _orient_outward(xyz, tri):
    """Flip triangles whose normal points toward the origin (star-shaped meshes)."""
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    flip = np.einsum("ij,ij->i", n, cen) < 0
    tri = tri.copy()
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return tri


def icosphere(level: int) -> Mesh:
    """Unit sphere: icosahedron refined `level` times (20*4**level triangles),
    every vertex projected onto radius 1."""
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    vlist = list(v)
    for _ in range(level):
        cache = {}
        nf = []

        def mid(i, j):
            key = (min(i, j), max(i, j))
            k = cache.get(key)
            if k is None:
                p = (vlist[i] + vlist[j]) / 2.0
                p = p / np.linalg.norm(p)
                vlist.append(p)
                k = len(vlist) - 1
                cache[key] = k
            return k

        for (i, j, k) in f:
            a, b, c = mid(i, j), mid(j, k), mid(k, i)
            nf += [(i, a, c), (j, b, a), (k, c, b), (a, b, c)]
        f = np.array(nf, dtype=np.int64)
    del verts
    xyz = np.array(vlist, dtype=np.float64)
    tri = _orient_outward(xyz, f)
    return Mesh(xyz, tri.astype(np.int32))


def ellipsoid(level: int, axes) -> Mesh:
    """Icosphere with vertices scaled by the semi-axes (a, b, c)."""
    m = icosphere(level)
    xyz = m.xyz * np.asarray(axes, dtype=np.float64)[None, :]
    return Mesh(xyz, _orient_outward(xyz, m.tri).astype(np.int32))


def rounded_cube(level: int, power: int = 8) -> Mesh:
    """Icosphere vertices projected radially onto |x|^p + |y|^p + |z|^p = 1."""
    m = icosphere(level)
    d = m.xyz
    s = np.sum(np.abs(d) ** power, axis=1) ** (-1.0 / power)
    xyz = d * s[:, None]
    return Mesh(xyz, _orient_outward(xyz, m.tri).astype(np.int32))


def torus(n_u: int, n_v: int, major: float = 1.0, minor: float = 0.3) -> Mesh:
    """Structured torus: n_u x n_v quads, each split into two triangles
    (2*n_u*n_v triangles), outward orientation."""
    u = 2.0 * np.pi * np.arange(n_u) / n_u
    v = 2.0 * np.pi * np.arange(n_v) / n_v
    U, V = np.meshgrid(u, v, indexing="ij")
    x = (major + minor * np.cos(V)) * np.cos(U)
    y = (major + minor * np.cos(V)) * np.sin(U)
    z = minor * np.sin(V)
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)

    def idx(i, j):
        return (i % n_u) * n_v + (j % n_v)

    tris = []
    for i in range(n_u):
        for j in range(n_v):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tris.append((a, b, c))
            tris.append((a, c, d))
    tri = np.array(tris, dtype=np.int64)
    # orient against the local tube centre (the torus is not star-shaped)
    A, B, C = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    nrm = np.cross(B - A, C - A)
    cen = (A + B + C) / 3.0
    phi = np.arctan2(cen[:, 1], cen[:, 0])
    core = np.stack([major * np.cos(phi), major * np.sin(phi), np.zeros_like(phi)], 1)
    flip = np.einsum("ij,ij->i", nrm, cen - core) < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return Mesh(xyz, tri.astype(np.int32))


def torus_for(nt: int) -> Mesh:
    """Torus with nt = 2*n_u*n_v triangles and n_u = 2.5*n_v (1280, 5120, 20480, ...)."""
    n_v = int(round(math.sqrt(nt / 5.0)))
    n_u = nt // (2 * n_v)
    assert 2 * n_u * n_v == nt, nt
    return torus(n_u, n_v)


def tetrahedron() -> Mesh:
    """Regular tetrahedron inscribed in the unit sphere (4 triangles)."""
    xyz = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    xyz /= math.sqrt(3.0)
    tri = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], dtype=np.int64)
    return Mesh(xyz, _orient_outward(xyz, tri).astype(np.int32))


def octahedron() -> Mesh:
    """Regular octahedron with vertices on the unit sphere (8 triangles)."""
    xyz = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                   dtype=np.float64)
    tri = []
    for a in (0, 1):
        for b in (2, 3):
            for c in (4, 5):
                tri.append((a, b, c))
    tri = np.array(tri, dtype=np.int64)
    return Mesh(xyz, _orient_outward(xyz, tri).astype(np.int32))


@dataclass
class Pulse:
    """Incident Gaussian plane-wave pulse u(x,t) = exp(-((t - delay - d.x)/width)^2)."""
    direction: np.ndarray
    width: float
    delay: float


def plane_wave_pulse(seed: int = SEED_BASE, width: float = 0.5,
                     direction=(0.0, 0.0, 1.0)) -> Pulse:
    """Pulse along `direction` with delay 1 + 4*width + U[0, width) drawn from the seed,
    so that the pulse is below exp(-16) on the unit ball at t = 0."""
    rng = np.random.default_rng(seed)
    delay = 1.0 + 4.0 * width + float(rng.uniform(0.0, width))
    d = np.asarray(direction, dtype=np.float64)
    return Pulse(d / np.linalg.norm(d), float(width), delay)


def mean_edge_length(m: Mesh) -> float:
    a, b, c = m.xyz[m.tri[:, 0]], m.xyz[m.tri[:, 1]], m.xyz[m.tri[:, 2]]
    e = np.concatenate([np.linalg.norm(b - a, axis=1), np.linalg.norm(c - b, axis=1),
                        np.linalg.norm(a - c, axis=1)])
    return float(e.mean())


# Named workloads: the parameter sets the tests and the benchmark run.
WORKLOADS = {
    # plain dense FP64 single layer on the 320-triangle sphere, BDF2, N=32
    "sphere320_N32": dict(level=2, N=32, dt=0.1, bdf=2),
    # compressed (H^2 + frequency ACA) single layer on the 5120-triangle sphere, N=256
    "sphere5120_N256": dict(level=4, N=256, dt=0.1, bdf=2),
}
