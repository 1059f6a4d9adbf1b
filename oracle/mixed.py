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


def p1_local(xyz, tri, I, J, s, qp: QuadParams = QuadParams()):
    """Local values of the triangle pairs (I[k] test, J[k] trial) at every
    frequency in s: K1 (ns, pairs, 3) over the trial triangle's vertices, Kp
    (ns, pairs, 3) over the test triangle's vertices, D (ns, pairs, 3, 3)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri)
    I = np.asarray(I, dtype=np.int64)
    J = np.asarray(J, dtype=np.int64)
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    ns = len(s)
    nrm = normals(xyz, tri)
    cu = curls(xyz, tri)
    K1l = np.zeros((ns, len(I), 3), dtype=np.complex128)
    Kpl = np.zeros((ns, len(I), 3), dtype=np.complex128)
    Dl = np.zeros((ns, len(I), 3, 3), dtype=np.complex128)
    for c, kk, X, Y, lx, ly, w in _pair_points(xyz, tri, I, J, qp):
        i, j = I[kk], J[kk]
        d = X - Y                                                  # x - y
        g, h = _kernels(d, s)                                      # (ns, pairs, points)
        dny = np.einsum("pqk,pk->pq", d, nrm[j])                  # (x - y) . n_y
        dnx = -np.einsum("pqk,pk->pq", d, nrm[i])                  # (y - x) . n_x
        # contractions over the points as batched products (pairs first)
        ht = np.moveaxis(h, 0, 1)                                  # (pairs, ns, points)
        kl = np.moveaxis(np.matmul(ht * (w * dny)[:, None, :], ly), 1, 0)   # (ns, pairs, 3)
        kpl = np.moveaxis(np.matmul(ht * (w * dnx)[:, None, :], lx), 1, 0)
        if c == 4:  # identical flat triangles: (x - y) . n = 0
            kl[:] = 0.0
            kpl[:] = 0.0
        gw = np.moveaxis(g, 0, 1) * w[:, None, :]                  # (pairs, ns, points)
        g0 = np.moveaxis(gw.sum(axis=2), 1, 0)                     # int int G: (ns, pairs)
        lxy = (lx[:, :, :, None] * ly[:, :, None, :]).reshape(lx.shape[0], lx.shape[1], 9)
        gl = np.moveaxis(np.matmul(gw, lxy), 1, 0).reshape(ns, lx.shape[0], 3, 3)  # int int G lx_a ly_b
        cc = np.einsum("pak,pbk->pab", cu[i], cu[j])               # curl . curl
        nn = np.einsum("pk,pk->p", nrm[i], nrm[j])
        K1l[:, kk] = kl
        Kpl[:, kk] = kpl
        Dl[:, kk] = g0[:, :, None, None] * cc[None] + (s ** 2)[:, None, None, None] * nn[None, :, None, None] * gl
    return K1l, Kpl, Dl


def _scatter(tri, nv, I, J, K1l, Kpl, Dl, out):
    """Adds the local values of the pairs (I, J) into out = (K1, Kp, D)."""
    tri = np.asarray(tri)
    K1, Kp, D = out
    for a in range(3):
        np.add.at(K1, (slice(None), I, tri[J, a]), K1l[:, :, a])
        np.add.at(Kp, (slice(None), tri[I, a], J), Kpl[:, :, a])
        for b in range(3):
            np.add.at(D, (slice(None), tri[I, a], tri[J, b]), Dl[:, :, a, b])


def p1_matrices(xyz, tri, s, qp: QuadParams = QuadParams()):
    """Dense K1 (len(s), M, nv), Kp (len(s), nv, M) and D (len(s), nv, nv)."""
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    M, nv, ns = len(tri), len(xyz), len(s)
    out = (np.zeros((ns, M, nv), dtype=np.complex128), np.zeros((ns, nv, M), dtype=np.complex128),
           np.zeros((ns, nv, nv), dtype=np.complex128))
    I, J = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")
    I = I.ravel()
    J = J.ravel()
    for k0 in range(0, len(I), 65536):
        sl = slice(k0, k0 + 65536)
        _scatter(tri, nv, I[sl], J[sl], *p1_local(xyz, tri, I[sl], J[sl], s, qp), out)
    return out


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


# ---- H^2 form (Sec. 4, eqs. degexp, uniformlr) of the P1 operators --------
# A far block b = r x c of triangle clusters carries, with the interpolation
# G(x - y) ~ sum_{mu, nu} L_{r,mu}(x) S_b[mu, nu] L_{c,nu}(y) (S_b of
# oracle.h2.coupling), the local values
#   K1 (test t in r, trial slot (t', a) in c):  U_r S_b W1_c^T,
#   Kp (test slot (t, a) in r, trial t' in c):  W1_r S_b U_c^T,
#   D  (slots (t, a) in r, (t', b) in c):       sum_k C_{r,k} S_b C_{c,k}^T + s^2 sum_k N_{r,k} S_b N_{c,k}^T,
# with the bases over the local vertex slots (t, a) of a cluster's triangles
#   W1[(t, a), nu] = int_t (n_t . grad L_nu) lambda_a,   U1[(t, a), nu] = int_t L_nu lambda_a,
#   C_k[(t, a), nu] = (curl lambda_a)_k int_t L_nu,      N_k[(t, a), nu] = n_{t,k} U1[(t, a), nu]
# (Radon's rule on each triangle, as for the P0 bases).  Near blocks keep the
# Galerkin values.

def p1_cluster_bases(xyz, tri, tree, c: int, m: int):
    """(W1, U1, C, N) of cluster c: W1, U1 (#c, 3, p); C, N (3, #c, 3, p) over
    the components k; triangles in the order of tree.indices(c)."""
    from .h2 import cheb_nodes, lagrange_1d, lagrange_3d
    from .dlayer import lagrange_1d_deriv
    P, area, _, _ = element_geometry(xyz, tri)
    nrm = normals(xyz, tri)
    cu = curls(xyz, tri)
    idx = tree.indices(c)
    nodes = cheb_nodes(tree.lo[c], tree.hi[c], m)
    X = np.einsum("qa,pad->pqd", Q.RADON7_BARY, P[idx]).reshape(-1, 3)
    p = m ** 3
    Lv = lagrange_3d(nodes, X).reshape(len(idx), 7, p)
    l = [lagrange_1d(nodes[a], X[:, a]) for a in range(3)]
    dl = [lagrange_1d_deriv(nodes[a], X[:, a]) for a in range(3)]
    g = [np.einsum("an,bn,cn->ncba", *(dl[k] if k == ax else l[k] for k in range(3))).reshape(len(X), p)
         for ax in range(3)]
    nrep = np.repeat(nrm[idx], 7, axis=0)
    dn = (nrep[:, 0:1] * g[0] + nrep[:, 1:2] * g[1] + nrep[:, 2:3] * g[2]).reshape(len(idx), 7, p)
    wb = Q.RADON7_W[:, None] * Q.RADON7_BARY                  # (7, 3): w_q lambda_a(q)
    W1 = area[idx][:, None, None] * np.einsum("qa,tqn->tan", wb, dn)
    U1 = area[idx][:, None, None] * np.einsum("qa,tqn->tan", wb, Lv)
    U0 = area[idx][:, None] * np.einsum("q,tqn->tn", Q.RADON7_W, Lv)
    C = np.einsum("tak,tn->ktan", cu[idx], U0)
    N = np.einsum("tk,tan->ktan", nrm[idx], U1)
    return W1, U1, C, N


def h2_p1_matrices(xyz, tri, s, tree, near, far, m: int, qp: QuadParams = QuadParams()):
    """H^2-expanded K1 (ns, M, nv), Kp (ns, nv, M), D (ns, nv, nv): near
    blocks of triangle clusters with the Galerkin values, far blocks with the
    interpolated kernel (module comment above)."""
    from .h2 import cluster_basis, coupling
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    tri = np.asarray(tri)
    M, nv, ns = len(tri), len(xyz), len(s)
    out = (np.zeros((ns, M, nv), dtype=np.complex128), np.zeros((ns, nv, M), dtype=np.complex128),
           np.zeros((ns, nv, nv), dtype=np.complex128))
    if len(near):
        I, J = [], []
        for r, c in near:
            a, b = np.meshgrid(tree.indices(r), tree.indices(c), indexing="ij")
            I.append(a.ravel())
            J.append(b.ravel())
        I = np.concatenate(I)
        J = np.concatenate(J)
        for k0 in range(0, len(I), 65536):
            sl = slice(k0, k0 + 65536)
            _scatter(tri, nv, I[sl], J[sl], *p1_local(xyz, tri, I[sl], J[sl], s, qp), out)
    cache = {}

    def bases(c):
        if c not in cache:
            cache[c] = (cluster_basis(xyz, tri, tree, c, m),) + p1_cluster_bases(xyz, tri, tree, c, m)
        return cache[c]

    K1, Kp, D = out
    for r, c in far:
        S = coupling(tree, r, c, s, m)                                  # (ns, p, p)
        Ur, W1r, _, Cr, Nr = bases(r)
        Uc, W1c, _, Cc, Nc = bases(c)
        ir, ic = tree.indices(r), tree.indices(c)
        k1 = np.einsum("tm,lmn,uan->ltua", Ur, S, W1c)                 # test t, trial slot (u, a)
        kp = np.einsum("tam,lmn,un->ltau", W1r, S, Uc)                 # test slot (t, a), trial u
        dd = (np.einsum("ktam,lmn,kubn->ltaub", Cr, S, Cc)
              + (s ** 2)[:, None, None, None, None] * np.einsum("ktam,lmn,kubn->ltaub", Nr, S, Nc))
        for a in range(3):
            np.add.at(K1, (slice(None), ir[:, None], tri[ic, a][None, :]), k1[:, :, :, a])
            np.add.at(Kp, (slice(None), tri[ir, a][:, None], ic[None, :]), kp[:, :, a, :])
            for b in range(3):
                np.add.at(D, (slice(None), tri[ir, a][:, None], tri[ic, b][None, :]), dd[:, :, a, :, b])
    return out
