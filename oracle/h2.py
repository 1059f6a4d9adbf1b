"""Chebyshev-interpolation H^2 bases and the H^2-expanded matrices (Sec. 4).

* eq. degexp / eq. uniformlr: far block b = r x c is approximated by
  U_r S_b W_c^H with U_r[i, mu] = int_{tau_i} L_{r,mu} dS and
  S_b[mu, nu] = g(xi_{r,mu}, xi_{c,nu}).  For P0 functions the bases are real,
  so W_c^H = U_c^T (row and column trees coincide).
* Def. 5 and Alg. 1: transfer matrices E_{r',r}[lambda, mu] = L_{r,mu}(xi_{r',lambda}).

Here U_r is computed DIRECTLY for every cluster (leaf or not) from r's own
Lagrange polynomials, never through transfer matrices, so that comparing with
a nested (transfer-based) implementation checks nestedness independently.

Readings: m first-kind Chebyshev points per axis, cos((2k+1) pi / (2m)),
k = 0..m-1, mapped to [lo, hi] of B_r by mid + half * x_k; a side of zero
extent gets half = 0.5e-8 * (box diagonal).  Multi-index flattening
mu = ix + m (iy + m iz).  Element integrals use Radon's 7-point rule.
"""
from __future__ import annotations

import numpy as np

from . import quadrature as Q
from .cluster import ClusterTree, box_diam
from .galerkin import FOUR_PI, QuadParams, element_geometry, pair_entries


def cheb_nodes(lo, hi, m: int):
    """(3, m) interpolation nodes of the box [lo, hi]."""
    k = np.arange(m)
    x = np.cos((2 * k + 1) * np.pi / (2 * m))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    mid = (lo + hi) * 0.5
    half = (hi - lo) * 0.5
    diag = float(box_diam(lo, hi))
    half = np.where(half > 0.0, half, 0.5e-8 * diag)
    return mid[:, None] + half[:, None] * x[None, :]


def lagrange_1d(nodes, t):
    """(m, n): l_k(t) = prod_{j != k} (t - t_j) / (t_k - t_j)."""
    m = len(nodes)
    t = np.asarray(t, dtype=np.float64)
    out = np.ones((m, len(t)))
    for k in range(m):
        for j in range(m):
            if j != k:
                out[k] *= (t - nodes[j]) / (nodes[k] - nodes[j])
    return out


def lagrange_3d(nodes3, X):
    """(n, m^3) values of the tensor Lagrange polynomials at points X (n, 3)."""
    m = nodes3.shape[1]
    lx = lagrange_1d(nodes3[0], X[:, 0])
    ly = lagrange_1d(nodes3[1], X[:, 1])
    lz = lagrange_1d(nodes3[2], X[:, 2])
    out = np.einsum("an,bn,cn->ncba", lx, ly, lz)          # index [n, iz, iy, ix]
    return out.reshape(len(X), m ** 3)


def tensor_points(nodes3):
    """(m^3, 3) interpolation points xi_mu with mu = ix + m (iy + m iz)."""
    m = nodes3.shape[1]
    iz, iy, ix = np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij")
    return np.stack([nodes3[0][ix.ravel()], nodes3[1][iy.ravel()], nodes3[2][iz.ravel()]], 1)


def cluster_basis(xyz, tri, tree: ClusterTree, r: int, m: int):
    """U_r (#r, m^3), rows in the order of tree.indices(r)."""
    P, area, _, _ = element_geometry(xyz, tri)
    idx = tree.indices(r)
    nodes = cheb_nodes(tree.lo[r], tree.hi[r], m)
    X = np.einsum("qa,pad->pqd", Q.RADON7_BARY, P[idx]).reshape(-1, 3)
    Lv = lagrange_3d(nodes, X).reshape(len(idx), 7, m ** 3)
    return area[idx][:, None] * np.einsum("q,pqm->pm", Q.RADON7_W, Lv)


def transfer(tree: ClusterTree, son: int, r: int, m: int):
    """E_{son,r}[lambda, mu] = L_{r,mu}(xi_{son,lambda})."""
    xs = tensor_points(cheb_nodes(tree.lo[son], tree.hi[son], m))
    return lagrange_3d(cheb_nodes(tree.lo[r], tree.hi[r], m), xs)


def coupling(tree: ClusterTree, r: int, c: int, s, m: int):
    """S_b[l, mu, nu] = exp(-s_l |xi_{c,nu} - xi_{r,mu}|) / (4 pi |xi_{c,nu} - xi_{r,mu}|)."""
    xr = tensor_points(cheb_nodes(tree.lo[r], tree.hi[r], m))
    xc = tensor_points(cheb_nodes(tree.lo[c], tree.hi[c], m))
    d = np.linalg.norm(xc[None, :, :] - xr[:, None, :], axis=2)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    return np.exp(-s[:, None, None] * d[None]) / (FOUR_PI * d[None])


def h2_matrices(xyz, tri, s, tree: ClusterTree, near, far, m: int,
                qp: QuadParams = QuadParams()):
    """H^2-expanded V_l (len(s), M, M) in the original triangle order:
    near blocks are Galerkin entries, far blocks U_r S_b(s_l) U_c^T."""
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    M = len(tri)
    out = np.zeros((len(s), M, M), dtype=np.complex128)
    if len(near):
        I, J = [], []
        for r, c in near:
            ir, ic = tree.indices(r), tree.indices(c)
            a, b = np.meshgrid(ir, ic, indexing="ij")
            I.append(a.ravel())
            J.append(b.ravel())
        I = np.concatenate(I)
        J = np.concatenate(J)
        e = pair_entries(xyz, tri, I, J, s, qp)
        out[:, I, J] = e.T
    cache = {}

    def U(r):
        if r not in cache:
            cache[r] = cluster_basis(xyz, tri, tree, r, m)
        return cache[r]

    for r, c in far:
        S = coupling(tree, r, c, s, m)
        blk = (U(r) @ S) @ U(c).T   # U_r S_b(s_l) U_c^T for every l (eq. uniformlr)
        out[:, tree.indices(r)[:, None], tree.indices(c)[None, :]] = blk
    return out
