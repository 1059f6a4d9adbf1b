"""Pins of the double-layer oracle and the direct Dirichlet formulation
(Sec. 2.2 eq. wavebio, Sec. 7.2 eq. cqmdir), against what the mathematics
fixes:

* Gauss's solid-angle identity: at s = 0, sum_j K[i, j] = -|tau_i| / 2 on a
  closed polyhedral surface (exactly, up to quadrature), on a sphere and an
  ellipsoid;
* the unit sphere: K 1 = mu_0(s) with mu_0(s) = 1/2 - (1 + s) e^{-s} sinh(s) / s
  (interior and exterior solutions i_0, k_0 of the modified Helmholtz
  equation and the jump of the double layer), O(h^2) with refinement;
* disjoint pairs against a high-order collapsed product rule;
* identical pairs vanish (flat triangles);
* the double-layer cluster basis reproduces n . grad p for polynomials of
  degree < m per axis; far blocks converge with m;
* the Dirichlet problem of a spherical wave from a source inside the sphere:
  the Neumann data of eq. cqmdir converge to the exact ones, and flipping the
  sign of K (a plausible mistake) does not.
"""
import numpy as np
import pytest

from oracle import cluster, cqm, dlayer, galerkin, h2
from oracle import quadrature as Q
from paper_2006_05186_gb300 import synth


def _mu0(s):
    return 0.5 - (1.0 + s) * np.exp(-s) * np.sinh(s) / s


@pytest.mark.parametrize("mesh", ["sphere", "ellipsoid"])
def test_gauss_identity(mesh):
    m = synth.icosphere(1) if mesh == "sphere" else synth.ellipsoid(1, (0.7, 1.0, 1.6))
    _, area, _, _ = galerkin.element_geometry(m.xyz, m.tri)
    K = dlayer.dense_dl_matrices(m.xyz, m.tri, [0.0])[0]
    assert np.max(np.abs(K.imag)) == 0.0
    err = np.max(np.abs(K.real.sum(axis=1) + 0.5 * area) / area)
    assert err < 5e-5, err
    # what is left is quadrature error: more singular points remove most of it
    K8 = dlayer.dense_dl_matrices(m.xyz, m.tri, [0.0], galerkin.QuadParams(g_sing=8))[0]
    err8 = np.max(np.abs(K8.real.sum(axis=1) + 0.5 * area) / area)
    assert err8 < 5e-7, (err, err8)


def test_identical_pairs_vanish():
    m = synth.icosphere(1)
    K = dlayer.dense_dl_matrices(m.xyz, m.tri, [1.0, 2.0 + 1.0j])
    assert np.all(np.diagonal(K, axis1=1, axis2=2) == 0.0)


def test_sphere_closed_form_converges():
    s = np.array([1.0, 3.0 + 2.0j])
    errs = []
    for level in (1, 2):
        m = synth.icosphere(level)
        _, area, _, _ = galerkin.element_geometry(m.xyz, m.tri)
        K = dlayer.dense_dl_matrices(m.xyz, m.tri, s)
        rows = K.sum(axis=2) / area[None, :]
        errs.append(np.max(np.abs(rows - _mu0(s)[:, None])))
    assert errs[1] < 3e-3 and errs[0] / errs[1] > 3.0, errs


def test_disjoint_pairs_against_a_fine_rule():
    m = synth.icosphere(2)
    P, area, cen, diam = galerkin.element_geometry(m.xyz, m.tri)
    nrm = dlayer.normals(m.xyz, m.tri)
    s = np.array([1.0, 2.0 + 4.0j])
    d = np.linalg.norm(cen - cen[0], axis=1)
    shared = np.array([len(set(m.tri[0]) & set(t)) for t in m.tri])
    ratio = d / np.maximum(diam, diam[0])
    j_near = int(np.argmin(np.where((shared == 0) & (ratio < 2.0), ratio, np.inf)))
    j_reg = int(np.argmin(np.where((shared == 0) & (ratio >= 2.0), ratio, np.inf)))
    bary, w = Q.collapsed_rule(16)
    for j in (j_near, j_reg):
        e = dlayer.dl_pair_entries(m.xyz, m.tri, [0], [j], s)[0]
        X = bary @ P[0]
        Y = bary @ P[j]
        dd = (X[:, None, :] - Y[None, :, :]).reshape(-1, 3)
        ww = area[0] * area[j] * (w[:, None] * w[None, :]).ravel()
        ref = dlayer._dl_kernel_sum(dd[None], nrm[j][None], ww[None], s)[0]
        err = np.max(np.abs(e - ref)) / np.max(np.abs(ref))
        assert err < (1e-7 if j == j_near else 5e-5), (j, err)


def test_cluster_basis_reproduces_normal_derivatives():
    m = synth.icosphere(2)
    t = cluster.build_tree(m.xyz, m.tri, 32)
    P, area, cen, _ = galerkin.element_geometry(m.xyz, m.tri)
    nrm = dlayer.normals(m.xyz, m.tri)
    c = 3
    mm = 4
    W = dlayer.dl_cluster_basis(m.xyz, m.tri, t, c, mm)
    xi = h2.tensor_points(h2.cheb_nodes(t.lo[c], t.hi[c], mm))
    idx = t.indices(c)
    a = np.array([0.3, -1.2, 0.7])
    lin = W @ (xi @ a)                                   # p = a.y
    assert np.allclose(lin, area[idx] * (nrm[idx] @ a), rtol=0, atol=1e-12)
    quad = W @ (xi[:, 0] * xi[:, 1])                     # p = y_x y_y: grad = (y_y, y_x, 0)
    ref = area[idx] * (nrm[idx, 0] * cen[idx, 1] + nrm[idx, 1] * cen[idx, 0])
    assert np.allclose(quad, ref, rtol=0, atol=1e-12)


def test_far_blocks_converge_with_m():
    m = synth.icosphere(2)
    t = cluster.build_tree(m.xyz, m.tri, 16)
    near, far = cluster.partition(t, 1.0)
    s = np.array([1.5])
    r, c = map(int, far[np.argmax([len(t.indices(b[0])) * len(t.indices(b[1])) for b in far])])
    I, J = np.meshgrid(t.indices(r), t.indices(c), indexing="ij")
    exact = dlayer.dl_pair_entries(m.xyz, m.tri, I.ravel(), J.ravel(), s)[:, 0].reshape(I.shape)
    errs = []
    for mm in (2, 3, 4):
        U = h2.cluster_basis(m.xyz, m.tri, t, r, mm)
        Wc = dlayer.dl_cluster_basis(m.xyz, m.tri, t, c, mm)
        approx = (U @ h2.coupling(t, r, c, s, mm)[0]) @ Wc.T
        errs.append(np.max(np.abs(approx - exact)) / np.max(np.abs(exact)))
    assert errs[2] < errs[1] / 4 < errs[0] / 16 and errs[2] < 0.03, errs


def _dirichlet_error(level, dt, N, flip=False):
    m = synth.icosphere(level)
    x0 = np.array([0.1, -0.2, 0.15])
    g, qex = dlayer.point_source(m.xyz, m.tri, N, dt, x0, 0.6, 2.5)
    K = None
    if flip:
        Ls = cqm.n_solved(N + 1)
        K = -dlayer.dense_dl_matrices(m.xyz, m.tri, cqm.frequencies(N, dt, 2)[:Ls])
    q, info = dlayer.solve_dirichlet(m.xyz, m.tri, N, dt, 2, g, K=K)
    assert info["max_imag"] < 1e-10
    return np.max(np.linalg.norm(q - qex, axis=1)) / np.max(np.linalg.norm(qex, axis=1))


def test_dirichlet_spherical_wave_converges():
    e1 = _dirichlet_error(1, 0.2, 24)
    e2 = _dirichlet_error(2, 0.1, 48)
    assert e2 < 0.035 and e1 / e2 > 3.0, (e1, e2)
    assert _dirichlet_error(1, 0.2, 24, flip=True) > 0.5
