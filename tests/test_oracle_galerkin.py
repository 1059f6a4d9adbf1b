"""Pins of the Galerkin assembly on the unit sphere: the single layer of the
Laplace-domain kernel (eq. fundsol) has the spherical harmonics as
eigenfunctions, lambda_0(s) = (1 - exp(-2s)) / (2s) and
lambda_1(s) = (s cosh s - sinh s)(1 + s) exp(-s) / s^3, and the flat-triangle
Galerkin approximation converges to them as O(h^2)."""
import numpy as np
import pytest

from oracle import galerkin as G
from oracle import quadrature as Q
from paper_2006_05186_gb300 import synth


def lam0(s):
    return (1.0 - np.exp(-2.0 * s)) / (2.0 * s)


def lam1(s):
    return (s * np.cosh(s) - np.sinh(s)) * (1.0 + s) * np.exp(-s) / s ** 3


S_TEST = [2.3 + 1.1j, 0.5 + 0.0j, 1.0 + 6.0j]


@pytest.fixture(scope="module")
def sphere_mats():
    out = {}
    for lev in (1, 2):
        m = synth.icosphere(lev)
        out[lev] = (m, G.dense_matrices(m.xyz, m.tri, np.array(S_TEST)))
    return out


def _rayleigh(m, V, phi):
    _, area, _, _ = G.element_geometry(m.xyz, m.tri)
    return (phi @ V @ phi) / (phi @ (area * phi))


def test_T3_l0_eigenvalue_converges(sphere_mats):
    for k, s in enumerate(S_TEST):
        errs = []
        for lev in (1, 2):
            m, V = sphere_mats[lev]
            one = np.ones(m.nt)
            errs.append(abs(_rayleigh(m, V[k], one) - lam0(s)) / abs(lam0(s)))
        assert errs[1] < 0.05 and errs[1] < errs[0] / 3.0, (s, errs)


def test_T3_l1_eigenvalue_converges(sphere_mats):
    for k, s in enumerate(S_TEST):
        errs = []
        for lev in (1, 2):
            m, V = sphere_mats[lev]
            _, _, cen, _ = G.element_geometry(m.xyz, m.tri)
            phi = cen[:, 2] / np.linalg.norm(cen, axis=1)
            errs.append(abs(_rayleigh(m, V[k], phi) - lam1(s)) / abs(lam1(s)))
        assert errs[1] < 0.05 and errs[1] < errs[0] / 3.0, (s, errs)


def test_T5_laplace_limit():
    m = synth.icosphere(2)
    V = G.dense_matrices(m.xyz, m.tri, np.array([1e-9 + 0j]))[0]
    _, area, _, _ = G.element_geometry(m.xyz, m.tri)
    assert abs(np.sum(V) / np.sum(area) - 1.0) < 0.02
    # eigenvalue 1/3 on Y_1
    _, _, cen, _ = G.element_geometry(m.xyz, m.tri)
    phi = cen[:, 2] / np.linalg.norm(cen, axis=1)
    assert abs(_rayleigh(m, V, phi) - 1.0 / 3.0) < 0.02


def test_matrix_symmetric_and_conjugate():
    """V(s) is complex symmetric (symmetric kernel, same test and trial space;
    every pair is evaluated in canonical order, so exactly); V(conj s) = conj V(s)."""
    m = synth.icosphere(1)
    s = 1.7 + 2.9j
    V = G.dense_matrices(m.xyz, m.tri, np.array([s, np.conj(s)]))
    assert np.max(np.abs(V[1] - np.conj(V[0]))) < 1e-15 * np.max(np.abs(V[0])) * 10
    assert np.array_equal(V[0], V[0].T)


def test_common_edge_rule_orders_agree_to_quadrature_accuracy():
    """The common-edge Sauter-Schwab rule applied with the two triangles
    exchanged gives the same entry up to the quadrature error: the canonical
    order chooses between two valid approximations, it does not hide a wrong
    rule.  Both orders also converge to each other as g grows."""
    m = synth.icosphere(1)
    tri = np.asarray(m.tri)
    pairs = [(i, j) for i in range(len(tri)) for j in range(len(tri))
             if i < j and len(set(tri[i]) & set(tri[j])) == 2][:12]
    s = np.array([0.8, 2.0 + 3.0j])
    P, _, _, _ = G.element_geometry(m.xyz, m.tri)

    def edge_entry(i, j, g):
        vx, vy = G._ordered_vertices(tri, i, j, 3)
        xh, yh, wr = Q.sauter_schwab("edge", g)
        X = Q.ref_to_bary(xh) @ np.asarray(m.xyz)[vx]
        Y = Q.ref_to_bary(yh) @ np.asarray(m.xyz)[vy]
        r = np.sqrt(np.sum((X - Y) ** 2, axis=1))
        area_i = 0.5 * np.linalg.norm(np.cross(P[i, 1] - P[i, 0], P[i, 2] - P[i, 0]))
        area_j = 0.5 * np.linalg.norm(np.cross(P[j, 1] - P[j, 0], P[j, 2] - P[j, 0]))
        w = wr * (2 * area_i) * (2 * area_j)
        return np.array([np.sum(w * np.exp(-sk * r) / (4 * np.pi * r)) for sk in s])

    for i, j in pairs:
        e5 = np.abs(edge_entry(i, j, 5) - edge_entry(j, i, 5)) / np.abs(edge_entry(i, j, 5))
        e9 = np.abs(edge_entry(i, j, 9) - edge_entry(j, i, 9)) / np.abs(edge_entry(i, j, 9))
        assert np.all(e5 < 1e-5) and np.all(e9 < e5 + 1e-13)


def test_T6_disjoint_pairs_brute_force():
    """Octahedron: opposite faces are disjoint; the production rule must agree
    with a high-order product rule (smooth integrand) to its own accuracy."""
    m = synth.octahedron()
    P, area, cen, diam = G.element_geometry(m.xyz, m.tri)
    s = np.array([0.8 + 3.0j])
    from oracle import quadrature as Q
    bary, w = Q.collapsed_rule(20)
    checked = 0
    for i in range(m.nt):
        for j in range(m.nt):
            if len(set(m.tri[i]) & set(m.tri[j])) == 0:
                X = bary @ P[i]
                Y = bary @ P[j]
                r = np.linalg.norm(X[:, None] - Y[None], axis=2)
                ref = area[i] * area[j] * np.sum(w[:, None] * w[None] * np.exp(-s[0] * r) / (4 * np.pi * r))
                got = G.pair_entries(m.xyz, m.tri, [i], [j], s)[0, 0]
                assert abs(got - ref) / abs(ref) < 1e-6
                checked += 1
    assert checked == 8


def test_classification_counts_icosphere():
    m = synth.icosphere(1)
    P, area, cen, diam = G.element_geometry(m.xyz, m.tri)
    I, J = np.meshgrid(np.arange(m.nt), np.arange(m.nt), indexing="ij")
    case = G.classify(m.tri, I.ravel(), J.ravel(), cen, diam, G.QuadParams())
    assert np.sum(case == 4) == m.nt
    assert np.sum(case == 3) == 3 * m.nt          # three edge neighbours each
    # each triangle shares a single vertex with (valence-3) triangles per vertex
    nv = m.nv
    val = np.bincount(m.tri.ravel(), minlength=nv)
    expect_vert = sum(int(val[a] - 3) for t in m.tri for a in t)
    assert np.sum(case == 2) == expect_vert
