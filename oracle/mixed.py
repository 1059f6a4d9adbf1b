"""Mixed boundary conditions with P1 elements: the operators and the solve of
Sec. 2.3 (eq. wavegalform) and Sec. 3.2 (eq. cqmgalapx), decoupled in
frequency like the single-layer solve.  Test infrastructure only: plain
numpy, FP64, dense matrices for small meshes.

Spaces: P0 (one constant per triangle) and P1 (one hat function per vertex;
on triangle t the hat of its vertex a is the barycentric coordinate
lambda_a).  The Laplace-domain operators at a frequency s, with the kernel
G(r) = exp(-s r) / (4 pi r), r = |x - y|, and flat triangles with unit
normals n = (P1 - P0) x (P2 - P0) / |...|:

* K1[m, v]  = <phi0_m, K phi1_v>, P0 test, P1 trial, kernel dG/dn_y =
  (x - y) . n_y (1 + s r) exp(-s r) / (4 pi r^3) (the double layer of
  oracle.dlayer with a P1 trial function);
* Kp[v, i]  = <phi1_v, K' phi0_i>, P1 test, P0 trial, kernel dG/dn_x =
  (y - x) . n_x (1 + s r) exp(-s r) / (4 pi r^3);
* D[u, v]   = <phi1_u, D phi1_v> in Maue's form,
  int int G(r) [curl phi1_u(x) . curl phi1_v(y) + s^2 (n_x . n_y) phi1_u(x) phi1_v(y)],
  curl = n x grad on the triangle, which for lambda_a is the opposite edge
  (P_{a+1} - P_{a+2}) / (2 |t|);
* I[m, v]   = <phi0_m, phi1_v> = |t_m| / 3 for v a vertex of t_m (P0 x P1
  mass), I' = I^T.

Quadrature: the rules of oracle.galerkin (Radon 7 x 7, collapsed Gauss for
near-singular pairs, Sauter-Schwab for pairs sharing vertices), test triangle
first; for the Sauter-Schwab pairs the barycentric coordinates of the rule
refer to the reordered vertices and are mapped back to each triangle's own
vertices.  Identical pairs contribute nothing to K1 and Kp ((x - y) . n = 0
on a flat triangle).

Mixed problem (eq. wavegalform, exterior problem): Gamma_D is a set of
triangles, Gamma_N the rest.  Unknowns: the Neumann data q on Gamma_D (P0)
and the Dirichlet data u on Gamma_N, in the hats of the vertices that touch
no Gamma_D triangle (so u vanishes on Gamma_D).  The data: g_D in P1 on the
vertices of Gamma_D's triangles (0 elsewhere), g_N in P0 on Gamma_N's
triangles (0 elsewhere).  Per solved frequency (hats: the R-scaled DFT of
oracle.cqm)
  V_DD q - K1_DN u = (-1/2 I + K1)_D: g_D - V_D: g_N,
  Kp_ND q + D_NN u = (-1/2 I' - Kp)_N: g_N - D_N: g_D,
solved by LU, then the inverse transform.
"""
from __future__ import annotations

import numpy as np

from . import cqm
from . import quadrature as Q
from .dense import fill_conjugate
from .dlayer import normals
from .galerkin import (QuadParams, _ordered_vertices, classify, dense_matrices,
                       element_geometry)

FOUR_PI = 4.0 * np.pi


def _kernels(d, s):
    """G(r) and (1 + s r) exp(-s r) / (4 pi r^3) for every s: (len(s), ...) each."""
    r = np.linalg.norm(d, axis=-1)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    e = np.exp(-s.reshape((-1,) + (1,) * r.ndim) * r[None])
    g = e / (FOUR_PI * r[None])
    h = (1.0 + s.reshape((-1,) + (1,) * r.ndim) * r[None]) * e / (FOUR_PI * r[None] ** 3)
    return g, h


def _pair_points(xyz, tri, I, J, qp: QuadParams, chunk: int = 2048):
    """Quadrature of the triangle pairs (I[k], J[k]), test triangle I[k]:
    yields (case, kk, X, Y, lx, ly, w) with points X (on I) and Y (on J) of shape
    (pairs, points, 3), the barycentric coordinates lx, ly of X and Y with
    respect to each triangle's stored vertices (pairs, points, 3) and the
    weights w (pairs, points), area factors included."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri)
    P, area, cen, diam = element_geometry(xyz, tri)
    case = classify(tri, I, J, cen, diam, qp)
    for c, (bary, wts) in ((0, (Q.RADON7_BARY, Q.RADON7_W)), (1, Q.collapsed_rule(qp.g_near))):
        idx = np.nonzero(case == c)[0]
        nq = len(wts)
        bx = np.repeat(bary, nq, axis=0)                  # point (p, q) -> x at p
        by = np.tile(bary, (nq, 1))                       # and y at q
        ww = (wts[:, None] * wts[None, :]).ravel()
        for k0 in range(0, len(idx), chunk):
            kk = idx[k0:k0 + chunk]
            X = bx @ P[I[kk]]
            Y = by @ P[J[kk]]
            w = (area[I[kk]] * area[J[kk]])[:, None] * ww[None, :]
            lx = np.broadcast_to(bx, (len(kk),) + bx.shape)
            ly = np.broadcast_to(by, (len(kk),) + by.shape)
            yield c, kk, X, Y, lx, ly, w
    for c, name in ((2, "vert"), (3, "edge"), (4, "ident")):
        idx = np.nonzero(case == c)[0]
        if len(idx) == 0:
            continue
        xh, yh, wr = Q.sauter_schwab(name, qp.g_sing)
        bx = Q.ref_to_bary(xh)
        by = Q.ref_to_bary(yh)
        sub = max(1, chunk // 32)
        for k0 in range(0, len(idx), sub):
            kk = idx[k0:k0 + sub]
            Px = np.empty((len(kk), 3, 3))
            Py = np.empty((len(kk), 3, 3))
            lx = np.empty((len(kk), len(wr), 3))
            ly = np.empty((len(kk), len(wr), 3))
            for t, k in enumerate(kk):
                vx, vy = _ordered_vertices(tri, I[k], J[k], c)
                Px[t] = xyz[vx]
                Py[t] = xyz[vy]
                # column a of the stored order is the rule's column vx.index(tri[I, a])
                lx[t] = bx[:, [vx.index(v) for v in tri[I[k]]]]
                ly[t] = by[:, [vy.index(v) for v in tri[J[k]]]]
            X = bx @ Px
            Y = by @ Py
            w = (4.0 * area[I[kk]] * area[J[kk]])[:, None] * wr[None, :]
            yield c, kk, X, Y, lx, ly, w


def curls(xyz, tri):
    """Surface curls of the three barycentric hats of every triangle:
    (M, 3, 3), [t, a] = (P_{a+1} - P_{a+2}) / (2 |t|)."""
    P, area, _, _ = element_geometry(xyz, tri)
    out = np.empty((len(tri), 3, 3))
    for a in range(3):
        out[:, a] = (P[:, (a + 1) % 3] - P[:, (a + 2) % 3]) / (2.0 * area[:, None])
    return out


def p1_matrices(xyz, tri, s, qp: QuadParams = QuadParams()):
    """Dense K1 (len(s), M, nv), Kp (len(s), nv, M) and D (len(s), nv, nv)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    M, nv, ns = len(tri), len(xyz), len(s)
    nrm = normals(xyz, tri)
    cu = curls(xyz, tri)
    I, J = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    I = I.ravel()
    J = J.ravel()
    K1 = np.zeros((ns, M, nv), dtype=np.complex128)
    Kp = np.zeros((ns, nv, M), dtype=np.complex128)
    D = np.zeros((ns, nv, nv), dtype=np.complex128)
    for c, kk, X, Y, lx, ly, w in _pair_points(xyz, tri, I, J, qp):
        i, j = I[kk], J[kk]
        d = X - Y                                                  # x - y
        g, h = _kernels(d, s)                                      # (ns, pairs, points)
        dny = np.einsum("pqk,pk->pq", d, nrm[j])                  # (x - y) . n_y
        dnx = -np.einsum("pqk,pk->pq", d, nrm[i])                  # (y - x) . n_x
        # contractions over the points as batched products (pairs first)
        ht = np.moveaxis(h, 0, 1)                                  # (pairs, ns, points)
        kl = np.moveaxis(np.matmul(ht * (w * dny)[:, None, :], ly), 1, 0)   # K1 local: (ns, pairs, 3)
        kpl = np.moveaxis(np.matmul(ht * (w * dnx)[:, None, :], lx), 1, 0)  # Kp local
        if c == 4:  # identical flat triangles: (x - y) . n = 0
            kl[:] = 0.0
            kpl[:] = 0.0
        gw = np.moveaxis(g, 0, 1) * w[:, None, :]                  # (pairs, ns, points)
        g0 = np.moveaxis(gw.sum(axis=2), 1, 0)                     # int int G: (ns, pairs)
        lxy = (lx[:, :, :, None] * ly[:, :, None, :]).reshape(lx.shape[0], lx.shape[1], 9)
        gl = np.moveaxis(np.matmul(gw, lxy), 1, 0).reshape(len(s), lx.shape[0], 3, 3)  # int int G lx_a ly_b
        cc = np.einsum("pak,pbk->pab", cu[i], cu[j])               # curl . curl
        nn = np.einsum("pk,pk->p", nrm[i], nrm[j])
        dl = g0[:, :, None, None] * cc[None] + (s ** 2)[:, None, None, None] * nn[None, :, None, None] * gl
        for a in range(3):
            va = tri[j, a]
            np.add.at(K1, (slice(None), i, va), kl[:, :, a])
            np.add.at(Kp, (slice(None), tri[i, a], j), kpl[:, :, a])
            for b in range(3):
                np.add.at(D, (slice(None), tri[i, a], tri[j, b]), dl[:, :, a, b])
    return K1, Kp, D


def mass_p0p1(xyz, tri):
    """I (M, nv): <phi0_m, phi1_v> = |t_m| / 3 for the vertices of t_m."""
    _, area, _, _ = element_geometry(xyz, tri)
    out = np.zeros((len(tri), len(xyz)))
    for a in range(3):
        np.add.at(out, (np.arange(len(tri)), np.asarray(tri)[:, a]), area / 3.0)
    return out


def mass_p1p1(xyz, tri):
    """(nv, nv): <phi1_u, phi1_v> = |t| (1 + delta_ab) / 12 summed over triangles."""
    _, area, _, _ = element_geometry(xyz, tri)
    tri = np.asarray(tri)
    out = np.zeros((len(xyz), len(xyz)))
    for a in range(3):
        for b in range(3):
            np.add.at(out, (tri[:, a], tri[:, b]), area * (2.0 if a == b else 1.0) / 12.0)
    return out


# ---- unit-sphere eigenvalues (modified spherical Bessel functions with
# i_0(z) = sinh z / z, k_0(z) = exp(-z) / z, so that exp(-s|x-y|)/(4 pi |x-y|)
# = s sum_n (2n+1)/(4 pi) i_n(s r<) k_n(s r>) P_n(cos gamma)) --------------

def sph_i(n, z):
    """i_n(z) for n = 0, 1 and its derivative."""
    z = np.asarray(z, dtype=np.complex128)
    i0 = np.sinh(z) / z
    i1 = (z * np.cosh(z) - np.sinh(z)) / z ** 2
    if n == 0:
        return i0, i1                       # i_0' = i_1
    return i1, i0 - 2.0 * i1 / z            # i_1' = i_0 - 2 i_1 / z


def sph_k(n, z):
    """k_n(z) for n = 0, 1 and its derivative."""
    z = np.asarray(z, dtype=np.complex128)
    k0 = np.exp(-z) / z
    k1 = np.exp(-z) * (z + 1.0) / z ** 2
    if n == 0:
        return k0, -k1                      # k_0' = -k_1
    return k1, -k0 - 2.0 * k1 / z           # k_1' = -k_0 - 2 k_1 / z


def sphere_eig_K(n, s):
    """Double layer on the unit sphere, K Y_n = (1/2 + s^2 i_n k_n') Y_n (the
    average of the interior and exterior limits of the potential)."""
    i, _ = sph_i(n, s)
    _, kp = sph_k(n, s)
    return 0.5 + s ** 2 * i * kp


def sphere_eig_D(n, s):
    """Hypersingular operator on the unit sphere, D Y_n = -s^3 i_n' k_n' Y_n
    (minus the normal derivative of the double-layer potential)."""
    _, ip = sph_i(n, s)
    _, kp = sph_k(n, s)
    return -(s ** 3) * ip * kp


# ---- the mixed problem ----------------------------------------------------

def mixed_spaces(tri, nv, dmask):
    """Triangles of Gamma_D (E_D), of Gamma_N (E_N), and the vertices of the
    Gamma_N space (V_N: no Gamma_D triangle touches them)."""
    tri = np.asarray(tri)
    dmask = np.asarray(dmask, dtype=bool)
    touch_d = np.zeros(nv, dtype=bool)
    touch_d[tri[dmask].ravel()] = True
    used = np.zeros(nv, dtype=bool)
    used[tri.ravel()] = True
    return np.nonzero(dmask)[0], np.nonzero(~dmask)[0], np.nonzero(used & ~touch_d)[0]


def solve_mixed(xyz, tri, N: int, dt: float, bdf: int, dmask, gD, gN, R: float | None = None,
                qp: QuadParams = QuadParams(), mats=None):
    """Neumann data q_n on Gamma_D (N+1, |E_D|) and Dirichlet data u_n on the
    Gamma_N space (N+1, |V_N|) of the mixed problem; gD (N+1, nv) P1
    coefficients (used on the vertices of Gamma_D's triangles), gN (N+1, M)
    P0 coefficients (used on Gamma_N's triangles).  mats: optional (V, K1,
    Kp, D) at the solved frequencies."""
    if R is None:
        R = cqm.default_R(N)
    L = N + 1
    Ls = cqm.n_solved(L)
    s = cqm.frequencies(N, dt, bdf, R)[:Ls]
    tri = np.asarray(tri)
    M, nv = len(tri), len(xyz)
    ED, EN, VN = mixed_spaces(tri, nv, dmask)
    if mats is None:
        V = dense_matrices(xyz, tri, s, qp)
        K1, Kp, D = p1_matrices(xyz, tri, s, qp)
    else:
        V, K1, Kp, D = mats
    Im = mass_p0p1(xyz, tri)
    gD = np.array(gD, dtype=np.float64)
    gN = np.array(gN, dtype=np.float64)
    keepD = np.zeros(nv, dtype=bool)
    keepD[tri[ED].ravel()] = True
    gD[:, ~keepD] = 0.0
    gN[:, ED] = 0.0
    gDh = cqm.forward(gD, R)[:Ls]
    gNh = cqm.forward(gN, R)[:Ls]
    nD, nN = len(ED), len(VN)
    qh = np.empty((Ls, nD), dtype=np.complex128)
    uh = np.empty((Ls, nN), dtype=np.complex128)
    for l in range(Ls):
        A = np.block([[V[l][np.ix_(ED, ED)], -K1[l][np.ix_(ED, VN)]],
                      [Kp[l][np.ix_(VN, ED)], D[l][np.ix_(VN, VN)]]])
        fD = (-0.5 * Im[ED] + K1[l][ED]) @ gDh[l] - V[l][ED] @ gNh[l]
        fN = (-0.5 * Im.T[VN] - Kp[l][VN]) @ gNh[l] - D[l][VN] @ gDh[l]
        x = np.linalg.solve(A, np.concatenate([fD, fN]))
        qh[l] = x[:nD]
        uh[l] = x[nD:]
    q = cqm.inverse(fill_conjugate(qh, L), R)
    u = cqm.inverse(fill_conjugate(uh, L), R)
    info = {"max_imag": float(max(np.max(np.abs(q.imag)), np.max(np.abs(u.imag)))),
            "ED": ED, "EN": EN, "VN": VN}
    return q.real, u.real, info


def point_source_vertices(xyz, N: int, dt: float, x0, width: float, delay: float):
    """Vertex values (N+1, nv) of the spherical wave u(x, t) = f(t - rho) /
    (4 pi rho), rho = |x - x0|, f(z) = exp(-((z - delay) / width)^2) (the
    field of oracle.dlayer.point_source, whose P0 Neumann data this pairs with)."""
    rho = np.linalg.norm(np.asarray(xyz, dtype=np.float64) - np.asarray(x0, dtype=np.float64)[None], axis=1)
    t = dt * np.arange(N + 1)
    z = (t[:, None] - rho[None] - delay) / width
    return np.exp(-z * z) / (FOUR_PI * rho[None])


def solve_mixed_mot(xyz, tri, N: int, dt: float, bdf: int, dmask, gD, gN, R: float | None = None,
                    qp: QuadParams = QuadParams(), mats_all=None):
    """The same mixed problem by the paper's own time stepping (Sec. 3.2, eqs.
    cqmgalapx and cqmrhs): the CQM weights Vhat_n, K1hat_n, Kphat_n, Dhat_n of
    the matrices at all L frequencies (eq. dft), and per step n the system
      [ Vhat_0,DD  -K1hat_0,DN ] [q_n]   [ -1/2 I_D: gD_n ]
      [ Kphat_0,ND  Dhat_0,NN  ] [u_n] = [ -1/2 I'_N: gN_n ]
          + sum_{k<=n} [ -Vhat_{n-k} gN_k + K1hat_{n-k} gD_k ; -Kphat_{n-k} gN_k - Dhat_{n-k} gD_k ]
          - sum_{k<n}  [ Vhat_{n-k} q_k - K1hat_{n-k} u_k ; Kphat_{n-k} q_k + Dhat_{n-k} u_k ],
    rows restricted to Gamma_D's triangles and Gamma_N's vertices, with one
    LU of the step matrix (a library primitive; the paper's Schur complement
    of Vhat_0 is the same elimination in two stages).  mats_all: optional
    (V, K1, Kp, D) at all L frequencies.  Returns (q, u, info) like
    solve_mixed; exactly causal, it differs from the decoupled solve by the
    wrap-around terms weighted by R^L."""
    from scipy.linalg import lu_factor, lu_solve
    from .mot import convolution_weights
    if R is None:
        R = cqm.default_R(N)
    L = N + 1
    s = cqm.frequencies(N, dt, bdf, R)
    tri = np.asarray(tri)
    M, nv = len(tri), len(xyz)
    ED, EN, VN = mixed_spaces(tri, nv, dmask)
    if mats_all is None:
        V = dense_matrices(xyz, tri, s, qp)
        K1, Kp, D = p1_matrices(xyz, tri, s, qp)
    else:
        V, K1, Kp, D = mats_all
    Vh, i1 = convolution_weights(V, R)
    K1h, i2 = convolution_weights(K1, R)
    Kph, i3 = convolution_weights(Kp, R)
    Dh, i4 = convolution_weights(D, R)
    Im = mass_p0p1(xyz, tri)
    gD = np.array(gD, dtype=np.float64)
    gN = np.array(gN, dtype=np.float64)
    keepD = np.zeros(nv, dtype=bool)
    keepD[tri[ED].ravel()] = True
    gD[:, ~keepD] = 0.0
    gN[:, ED] = 0.0
    nD, nN = len(ED), len(VN)
    A0 = np.block([[Vh[0][np.ix_(ED, ED)], -K1h[0][np.ix_(ED, VN)]],
                   [Kph[0][np.ix_(VN, ED)], Dh[0][np.ix_(VN, VN)]]])
    lu = lu_factor(A0)
    q = np.zeros((L, nD))
    u = np.zeros((L, nN))
    for n in range(L):
        fD = -0.5 * Im[ED] @ gD[n]
        fN = -0.5 * Im.T[VN] @ gN[n]
        for k in range(n + 1):
            fD += -Vh[n - k][ED] @ gN[k] + K1h[n - k][ED] @ gD[k]
            fN += -Kph[n - k][VN] @ gN[k] - Dh[n - k][VN] @ gD[k]
        for k in range(n):
            fD -= Vh[n - k][np.ix_(ED, ED)] @ q[k] - K1h[n - k][np.ix_(ED, VN)] @ u[k]
            fN -= Kph[n - k][np.ix_(VN, ED)] @ q[k] + Dh[n - k][np.ix_(VN, VN)] @ u[k]
        x = lu_solve(lu, np.concatenate([fD, fN]))
        q[n] = x[:nD]
        u[n] = x[nD:]
    return q, u, {"imag_rel": max(i1, i2, i3, i4), "ED": ED, "EN": EN, "VN": VN}
