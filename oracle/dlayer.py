"""P0 Galerkin double layer of the Laplace-domain kernel and the direct
formulation of the sound-soft (Dirichlet) problem.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* The double layer (Sec. 2.2, eq. wavebio: K with the kernel gamma_{1,y} of
  the fundamental solution) in the Laplace domain, P0 test and trial functions:
      K_l[i, j] = int_{tau_i} int_{tau_j} d/dn_y [exp(-s_l r) / (4 pi r)] dS_y dS_x
                = int int (x - y).n_j (1 + s_l r) exp(-s_l r) / (4 pi r^3),
  r = |x - y|, n_j the unit normal of tau_j (vertices counter-clockwise seen
  from outside: the outward normal).
* Quadrature as for the single layer (galerkin.py: classification, rules and
  the vertex order of the singular rules), but the pair is NOT swapped into
  canonical order: the kernel is not symmetric, and (i, j) is always (test,
  trial).  Reading: on a flat triangle (x - y).n_j vanishes identically, so
  K_l[i, i] = 0.
* Far blocks (Sec. 4 with the remark after Thm. 1 on the double layer):
  interpolating the kernel in x and y and differentiating the y-interpolant,
      K_l|_b ~ U_r S_b(s_l) W_c^T,  W_c[j, nu] = int_{tau_j} n_j . grad L_{c,nu}(y) dS_y,
  with the same couplings S_b as the single layer.  W_c is computed here
  directly from c's own Lagrange polynomials (Radon's 7-point rule).
* The direct formulation of the Dirichlet problem (Sec. 7.2, eq. cqmdir),
  decoupled in frequency as in the Remark of Sec. 6.2:
      V_l qhat_l = (-1/2 M + K_l) ghat_l,   M = diag |tau_i| (P0 mass matrix),
  ghat_l = sum_n R^n g_n zeta^{nl} with g_n the P0 (L^2-projection)
  coefficients of the Dirichlet data at t_n; q_n from the inverse transform.
"""
from __future__ import annotations

import numpy as np

from . import cqm
from . import quadrature as Q
from .cluster import ClusterTree
from .dense import fill_conjugate
from .galerkin import FOUR_PI, QuadParams, _ordered_vertices, classify, element_geometry
from .h2 import cheb_nodes, coupling, lagrange_1d


def normals(xyz, tri):
    """Unit normals (M, 3) of the triangles, (P1 - P0) x (P2 - P0) normalised."""
    P = np.asarray(xyz, dtype=np.float64)[np.asarray(tri)]
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    return n / np.linalg.norm(n, axis=1)[:, None]


def _dl_kernel_sum(d, nj, w, s):
    """sum_k w_k (d_k . n) (1 + s r_k) exp(-s r_k) / (4 pi r_k^3) along the
    point axis; d: (..., points, 3) = x - y, nj: (..., 3)."""
    r = np.linalg.norm(d, axis=-1)
    dn = np.einsum("...pk,...k->...p", d, nj)
    c = w * dn / (FOUR_PI * r ** 3)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    out = np.empty(r.shape[:-1] + (len(s),), dtype=np.complex128)
    for k, sk in enumerate(s):
        out[..., k] = np.sum(c * (1.0 + sk * r) * np.exp(-sk * r), axis=-1)
    return out


def dl_pair_entries(xyz, tri, I, J, s, qp: QuadParams = QuadParams(), chunk: int = 4096):
    """Double-layer entries K[I[k], J[k]] at every frequency in s: (len(I), len(s))."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri)
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    P, area, cen, diam = element_geometry(xyz, tri)
    nrm = normals(xyz, tri)
    case = classify(tri, I, J, cen, diam, qp)
    out = np.zeros((len(I), len(s)), dtype=np.complex128)
    for c, (bary, wts) in ((0, (Q.RADON7_BARY, Q.RADON7_W)), (1, Q.collapsed_rule(qp.g_near))):
        idx = np.nonzero(case == c)[0]
        ww = (wts[:, None] * wts[None, :]).ravel()
        for k0 in range(0, len(idx), chunk):
            kk = idx[k0:k0 + chunk]
            X = bary @ P[I[kk]]
            Y = bary @ P[J[kk]]
            d = (X[:, :, None, :] - Y[:, None, :, :]).reshape(len(kk), -1, 3)
            w = (area[I[kk]] * area[J[kk]])[:, None] * ww[None, :]
            out[kk] = _dl_kernel_sum(d, nrm[J[kk]], w, s)
    for c, name in ((2, "vert"), (3, "edge")):  # identical pairs stay 0
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
            d = bx @ Px - by @ Py
            w = (4.0 * area[I[kk]] * area[J[kk]])[:, None] * wr[None, :]
            out[kk] = _dl_kernel_sum(d, nrm[J[kk]], w, s)
    return out


def dense_dl_matrices(xyz, tri, s, qp: QuadParams = QuadParams()):
    """Dense K_l for every frequency in s: complex (len(s), M, M)."""
    M = len(tri)
    I, J = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    e = dl_pair_entries(xyz, tri, I.ravel(), J.ravel(), s, qp)
    return np.moveaxis(e.reshape(M, M, -1), 2, 0)


def lagrange_1d_deriv(nodes, t):
    """(m, n): l_k'(t) = sum_{i != k} 1/(t_k - t_i) prod_{j != k, i} (t - t_j)/(t_k - t_j)."""
    m = len(nodes)
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros((m, len(t)))
    for k in range(m):
        for i in range(m):
            if i == k:
                continue
            term = np.full(len(t), 1.0 / (nodes[k] - nodes[i]))
            for j in range(m):
                if j != k and j != i:
                    term *= (t - nodes[j]) / (nodes[k] - nodes[j])
            out[k] += term
    return out


def dl_cluster_basis(xyz, tri, tree: ClusterTree, c: int, m: int):
    """W_c (#c, m^3): int_{tau_j} n_j . grad L_{c,nu} dS (Radon 7 points), rows in
    the order of tree.indices(c); nu = ix + m (iy + m iz)."""
    P, area, _, _ = element_geometry(xyz, tri)
    nrm = normals(xyz, tri)
    idx = tree.indices(c)
    nodes = cheb_nodes(tree.lo[c], tree.hi[c], m)
    X = np.einsum("qa,pad->pqd", Q.RADON7_BARY, P[idx]).reshape(-1, 3)
    l = [lagrange_1d(nodes[a], X[:, a]) for a in range(3)]
    dl = [lagrange_1d_deriv(nodes[a], X[:, a]) for a in range(3)]
    # gradient components, index [point, iz, iy, ix]
    gx = np.einsum("an,bn,cn->ncba", dl[0], l[1], l[2]).reshape(len(X), m ** 3)
    gy = np.einsum("an,bn,cn->ncba", l[0], dl[1], l[2]).reshape(len(X), m ** 3)
    gz = np.einsum("an,bn,cn->ncba", l[0], l[1], dl[2]).reshape(len(X), m ** 3)
    nrep = np.repeat(nrm[idx], 7, axis=0)
    dn = (nrep[:, 0:1] * gx + nrep[:, 1:2] * gy + nrep[:, 2:3] * gz).reshape(len(idx), 7, m ** 3)
    return area[idx][:, None] * np.einsum("q,pqm->pm", Q.RADON7_W, dn)


def h2_dl_matrices(xyz, tri, s, tree: ClusterTree, near, far, m: int,
                   qp: QuadParams = QuadParams()):
    """H^2-expanded K_l (len(s), M, M): near blocks are Galerkin entries, far
    blocks U_r S_b(s_l) W_c^T."""
    from .h2 import cluster_basis
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    M = len(tri)
    out = np.zeros((len(s), M, M), dtype=np.complex128)
    if len(near):
        I, J = [], []
        for r, c in near:
            a, b = np.meshgrid(tree.indices(r), tree.indices(c), indexing="ij")
            I.append(a.ravel())
            J.append(b.ravel())
        I = np.concatenate(I)
        J = np.concatenate(J)
        out[:, I, J] = dl_pair_entries(xyz, tri, I, J, s, qp).T
    for r, c in far:
        S = coupling(tree, r, c, s, m)
        U = cluster_basis(xyz, tri, tree, r, m)
        W = dl_cluster_basis(xyz, tri, tree, c, m)
        out[:, tree.indices(r)[:, None], tree.indices(c)[None, :]] = (U @ S) @ W.T
    return out


def dirichlet_rhs(K, area, ghat):
    """(-1/2 M + K_l) ghat_l for every l: K (Ls, M, M), ghat (Ls, M)."""
    return -0.5 * area[None, :] * ghat + np.einsum("lij,lj->li", K, ghat)


def solve_dirichlet(xyz, tri, N: int, dt: float, bdf: int, g, R: float | None = None,
                    V=None, K=None, qp: QuadParams = QuadParams()):
    """Neumann data q_n (N+1, M) of the Dirichlet problem with P0 data
    coefficients g (N+1, M): eq. cqmdir decoupled in frequency, one LU per
    solved frequency (V and K: the (Ls, M, M) matrices of the solved
    frequencies, dense Galerkin when not given)."""
    from .galerkin import dense_matrices
    if R is None:
        R = cqm.default_R(N)
    L = N + 1
    Ls = cqm.n_solved(L)
    s = cqm.frequencies(N, dt, bdf, R)[:Ls]
    if V is None:
        V = dense_matrices(xyz, tri, s, qp)
    if K is None:
        K = dense_dl_matrices(xyz, tri, s, qp)
    _, area, _, _ = element_geometry(xyz, tri)
    ghat = cqm.forward(np.asarray(g, dtype=np.float64), R)[:Ls]
    rhs = dirichlet_rhs(K, area, ghat)
    qhat = np.stack([np.linalg.solve(V[l], rhs[l]) for l in range(Ls)])
    q = cqm.inverse(fill_conjugate(qhat, L), R)
    return q.real, {"qhat": qhat, "max_imag": float(np.max(np.abs(q.imag)))}


def point_source(xyz, tri, N: int, dt: float, x0, width: float, delay: float):
    """P0 coefficients of the Dirichlet and Neumann traces of the spherical wave
    u(x, t) = f(t - rho) / (4 pi rho), rho = |x - x0|, f(z) = exp(-((z - delay)/width)^2),
    a solution of the wave equation away from x0 (Sec. 7.2 uses a spherical
    wave of this form as its exact solution):
    g_n[i] = (1/|tau_i|) int_{tau_i} u(., t_n),  q_n[i] = (1/|tau_i|) int_{tau_i} du/dn(., t_n),
    Radon's 7-point rule, n the outward unit normal."""
    P, area, _, _ = element_geometry(xyz, tri)
    nrm = normals(xyz, tri)
    X = np.einsum("qa,pad->pqd", Q.RADON7_BARY, P)            # (M, 7, 3)
    d = X - np.asarray(x0, dtype=np.float64)[None, None, :]
    rho = np.linalg.norm(d, axis=2)
    dn = np.einsum("pqk,pk->pq", d, nrm) / rho                 # d rho / dn
    t = dt * np.arange(N + 1)
    g = np.empty((N + 1, len(tri)))
    q = np.empty((N + 1, len(tri)))
    for n, tn in enumerate(t):
        z = (tn - rho - delay) / width
        f = np.exp(-z * z)
        fp = -2.0 * z / width * f                              # f'(t - rho)
        u = f / (FOUR_PI * rho)
        # du/dn = (-f'/rho - f/rho^2) / (4 pi) * d rho / dn
        un = (-fp / rho - f / rho ** 2) / FOUR_PI * dn
        g[n] = u @ Q.RADON7_W
        q[n] = un @ Q.RADON7_W
    return g, q
