"""P0 Galerkin entries of the Laplace-domain single layer (Sec. 3.2).

V_l[i, j] = int_{tau_i} int_{tau_j} exp(-s_l |x - y|) / (4 pi |x - y|) dS_y dS_x
(eq. fundsol and the Galerkin matrices of Sec. 3.2, P0 test and trial
functions on flat triangles).

Reading of the quadrature, which the paper leaves open (the same rule set is
specified for the CUDA path):
* a pair is classified by shared vertex indices: 3 -> identical, 2 -> common
  edge, 1 -> common vertex (Sauter-Schwab, g_sing^4 points per region);
* a pair with no shared vertex is near-singular when the distance of the
  centroids is below near_ratio * max(longest edge of tau_i, of tau_j): the
  collapsed Gauss rule with g_near^2 points on each triangle (centroids as
  ((P0 + P1) + P2) / 3, lengths as sqrt((x^2 + y^2) + z^2), so that the
  decision is reproducible bit for bit);
* otherwise regular: Radon's 7-point rule on each triangle (49 points).
Every pair is evaluated in canonical order, the lower triangle index first:
V[i, j] for i > j is the rule applied to (j, i).  The kernel is symmetric and
test and trial spaces coincide, so the Galerkin matrix is symmetric (Sec. 3.2);
the common-edge rule is not symmetric under exchanging the two triangles (its
two orders differ by the quadrature error, ~4e-7 relative at g_sing = 5), and
the canonical order makes the discrete matrix exactly symmetric.
Vertex order used by the singular rules (pair i = test, j = trial, i <= j):
* identical: the stored order (v0, v1, v2) on both sides;
* common edge: (u, w, third) on both sides, where (u, w) are the shared
  vertices in the order they appear in triangle i;
* common vertex: each triangle rotated cyclically to start at the shared
  vertex.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import quadrature as Q

FOUR_PI = 4.0 * np.pi


@dataclass(frozen=True)
class QuadParams:
    g_sing: int = 5
    g_near: int = 5
    near_ratio: float = 2.0


def element_geometry(xyz, tri):
    """Per-triangle vertices (M,3,3), area, centroid, longest edge."""
    P = np.asarray(xyz, dtype=np.float64)[np.asarray(tri)]
    e01 = P[:, 1] - P[:, 0]
    e02 = P[:, 2] - P[:, 0]
    cr = np.cross(e01, e02)
    area = 0.5 * np.sqrt(np.sum(cr * cr, axis=1))
    cen = (P[:, 0] + P[:, 1] + P[:, 2]) / 3.0
    l0 = _length(P[:, 1] - P[:, 0])
    l1 = _length(P[:, 2] - P[:, 1])
    l2 = _length(P[:, 0] - P[:, 2])
    diam = np.maximum(np.maximum(l0, l1), l2)
    return P, area, cen, diam


def _length(d):
    """Euclidean length with the sum formed as ((x^2 + y^2) + z^2)."""
    return np.sqrt((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2])


def classify(tri, I, J, cen, diam, qp: QuadParams):
    """Case per pair: 0 regular, 1 near-singular, 2 common vertex, 3 common edge, 4 identical."""
    tri = np.asarray(tri)
    A = tri[I]
    B = tri[J]
    shared = np.zeros(len(I), dtype=np.int64)
    for a in range(3):
        for b in range(3):
            shared += (A[:, a] == B[:, b])
    case = np.zeros(len(I), dtype=np.int64)
    d = _length(cen[I] - cen[J])
    near = d < qp.near_ratio * np.maximum(diam[I], diam[J])
    case[(shared == 0) & near] = 1
    case[shared == 1] = 2
    case[shared == 2] = 3
    case[shared == 3] = 4
    return case


def _ordered_vertices(tri, i, j, case):
    """Vertex index triples (P_x, P_y) for a singular pair, per the module docstring."""
    ti = list(tri[i])
    tj = list(tri[j])
    if case == 4:
        return ti, ti
    if case == 3:
        sh = [v for v in ti if v in tj]
        u, w = sh[0], sh[1]
        oi = [v for v in ti if v not in sh][0]
        oj = [v for v in tj if v not in sh][0]
        return [u, w, oi], [u, w, oj]
    if case == 2:
        u = [v for v in ti if v in tj][0]
        ki = ti.index(u)
        kj = tj.index(u)
        return ti[ki:] + ti[:ki], tj[kj:] + tj[:kj]
    raise ValueError(case)


def _kernel_sum(r, w, s):
    """sum_k w_k exp(-s r_k) / (4 pi r_k) along the last axis, for each s."""
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    out = np.empty(r.shape[:-1] + (len(s),), dtype=np.complex128)
    for k, sk in enumerate(s):
        out[..., k] = np.sum(w * np.exp(-sk * r) / (FOUR_PI * r), axis=-1)
    return out


def pair_entries(xyz, tri, I, J, s, qp: QuadParams = QuadParams(), chunk: int = 4096):
    """Galerkin entries V[I[k], J[k]] at every frequency in s: complex (len(I), len(s))."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri)
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    I, J = np.minimum(I, J), np.maximum(I, J)  # canonical order (module docstring)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    P, area, cen, diam = element_geometry(xyz, tri)
    case = classify(tri, I, J, cen, diam, qp)
    out = np.zeros((len(I), len(s)), dtype=np.complex128)

    # regular and near-singular pairs: product of triangle rules
    for c, (bary, wts) in ((0, (Q.RADON7_BARY, Q.RADON7_W)), (1, Q.collapsed_rule(qp.g_near))):
        idx = np.nonzero(case == c)[0]
        ww = (wts[:, None] * wts[None, :]).ravel()
        for k0 in range(0, len(idx), chunk):
            kk = idx[k0:k0 + chunk]
            X = bary @ P[I[kk]]   # (pairs, points, xyz): sum_a bary[q, a] P[p, a]
            Y = bary @ P[J[kk]]
            r = np.linalg.norm(X[:, :, None, :] - Y[:, None, :, :], axis=3).reshape(len(kk), -1)
            w = (area[I[kk]] * area[J[kk]])[:, None] * ww[None, :]
            out[kk] = _kernel_sum(r, w, s)

    # singular pairs: Sauter-Schwab
    for c, name in ((2, "vert"), (3, "edge"), (4, "ident")):
        idx = np.nonzero(case == c)[0]
        if len(idx) == 0:
            continue
        xh, yh, wr = Q.sauter_schwab(name, qp.g_sing)
        bx = Q.ref_to_bary(xh)
        by = Q.ref_to_bary(yh)
        sub = max(1, chunk // 16)
        for k0 in range(0, len(idx), sub):
            kk = idx[k0:k0 + sub]
            Px = np.empty((len(kk), 3, 3))
            Py = np.empty((len(kk), 3, 3))
            for t, k in enumerate(kk):
                vx, vy = _ordered_vertices(tri, I[k], J[k], c)
                Px[t] = xyz[vx]
                Py[t] = xyz[vy]
            X = bx @ Px
            Y = by @ Py
            r = np.linalg.norm(X - Y, axis=2)
            w = (4.0 * area[I[kk]] * area[J[kk]])[:, None] * wr[None, :]
            out[kk] = _kernel_sum(r, w, s)
    return out


def dense_matrices(xyz, tri, s, qp: QuadParams = QuadParams()):
    """Dense V_l for every frequency in s: complex (len(s), M, M)."""
    M = len(tri)
    I, J = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    e = pair_entries(xyz, tri, I.ravel(), J.ravel(), s, qp)
    return np.moveaxis(e.reshape(M, M, -1), 2, 0)
