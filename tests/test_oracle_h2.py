"""Pins of the Chebyshev-interpolation H^2 oracle (Sec. 4.2, Def. 5, Thm. 1):
polynomial reproduction, nestedness, error decay in the order m."""
import numpy as np
import pytest

from oracle import cluster, cqm, galerkin as G, h2, quadrature as Q
from paper_2006_05186_gb300 import synth


@pytest.fixture(scope="module")
def setup1280():
    m = synth.icosphere(3)
    t = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t, 1.0)
    return m, t, near, far


def test_lagrange_cardinal_and_partition_of_unity():
    nodes = h2.cheb_nodes([0, 0, 0], [1, 2, 3], 4)
    pts = h2.tensor_points(nodes)
    Lv = h2.lagrange_3d(nodes, pts)
    assert np.allclose(Lv, np.eye(64), atol=1e-13)
    X = np.random.default_rng(0).uniform(0, 1, (50, 3)) * [1, 2, 3]
    assert np.allclose(h2.lagrange_3d(nodes, X).sum(1), 1.0, atol=1e-12)


def test_T8_polynomial_reproduction(setup1280):
    """A kernel of degree < m per coordinate is reproduced exactly by
    U_r S_b U_c^T (both sides use the same element rule)."""
    m, t, near, far = setup1280
    P, area, _, _ = G.element_geometry(m.xyz, m.tri)
    poly = lambda x, y: (1.0 + x[..., 0] * y[..., 1] - 0.5 * x[..., 2] * y[..., 2]) ** 2 * (2.0 + x[..., 1] ** 3) * (1 + y[..., 0])
    r, c = far[len(far) // 2]
    mm = 4
    Ur = h2.cluster_basis(m.xyz, m.tri, t, r, mm)
    Uc = h2.cluster_basis(m.xyz, m.tri, t, c, mm)
    xr = h2.tensor_points(h2.cheb_nodes(t.lo[r], t.hi[r], mm))
    xc = h2.tensor_points(h2.cheb_nodes(t.lo[c], t.hi[c], mm))
    S = poly(xr[:, None, :], xc[None, :, :])
    approx = Ur @ S @ Uc.T
    X = np.einsum("qa,pad->pqd", Q.RADON7_BARY, P)
    ir, ic = t.indices(r), t.indices(c)
    ref = np.einsum("i,j,p,q,ipjq->ij", area[ir], area[ic], Q.RADON7_W, Q.RADON7_W,
                    poly(X[ir][:, :, None, None, :], X[ic][None, None, :, :, :]))
    assert np.max(np.abs(approx - ref)) < 1e-12 * np.max(np.abs(ref))


def test_T8_nestedness(setup1280):
    m, t, _, _ = setup1280
    for r in range(t.n_nodes):
        if t.is_leaf(r):
            continue
        Ur = h2.cluster_basis(m.xyz, m.tri, t, r, 4)
        off = 0
        for son in t.sons[r]:
            Us = h2.cluster_basis(m.xyz, m.tri, t, son, 4)
            E = h2.transfer(t, son, r, 4)
            n = len(t.indices(son))
            assert np.max(np.abs(Ur[off:off + n] - Us @ E)) < 1e-12 * np.max(np.abs(Ur))
            off += n


def test_T8_interpolation_error_decays_with_order(setup1280):
    """Thm. 1: the far-block error falls geometrically with m."""
    m, t, near, far = setup1280
    s = np.array([1.5 + 4.0j])
    blocks = far[:: max(1, len(far) // 12)]
    errs = []
    for mm in (2, 3, 4, 5):
        num = den = 0.0
        for r, c in blocks:
            ir, ic = t.indices(r), t.indices(c)
            I, J = np.meshgrid(ir, ic, indexing="ij")
            ref = G.pair_entries(m.xyz, m.tri, I.ravel(), J.ravel(), s)[:, 0].reshape(len(ir), len(ic))
            Ur = h2.cluster_basis(m.xyz, m.tri, t, r, mm)
            Uc = h2.cluster_basis(m.xyz, m.tri, t, c, mm)
            S = h2.coupling(t, r, c, s, mm)[0]
            num += np.sum(np.abs(Ur @ S @ Uc.T - ref) ** 2)
            den += np.sum(np.abs(ref) ** 2)
        errs.append(np.sqrt(num / den))
    assert all(errs[k + 1] < errs[k] / 1.5 for k in range(3)), errs
    assert errs[2] < 1e-2, errs


def test_h2_expanded_matches_dense_on_near_field_and_approximates_far():
    m = synth.icosphere(2)
    t = cluster.build_tree(m.xyz, m.tri, 16)
    near, far = cluster.partition(t, 1.0)
    assert len(far) > 0
    s = np.array([2.0 + 3.0j])
    Vh = h2.h2_matrices(m.xyz, m.tri, s, t, near, far, 4)[0]
    Vd = G.dense_matrices(m.xyz, m.tri, s)[0]
    mask = np.zeros_like(Vd, dtype=bool)
    for r, c in near:
        mask[np.ix_(t.indices(r), t.indices(c))] = True
    assert np.array_equal(Vh[mask], Vd[mask])
    rel = np.linalg.norm(Vh - Vd) / np.linalg.norm(Vd)
    assert 0 < rel < 1e-2


def test_pool_assembly_equals_serial():
    """The process-pool evaluation of the H^2-expanded matrices is the serial
    oracle bit for bit (it only evaluates independent pairs and blocks in
    different processes), and its per-frequency LU solve is LAPACK's."""
    from oracle import pool
    m = synth.icosphere(2)
    t = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t, 1.0)
    s = cqm.frequencies(16, 0.1, 2)[[0, 5]]
    V = h2.h2_matrices(m.xyz, m.tri, s, t, near, far, 4)
    Vp = pool.h2_matrices(m.xyz, m.tri, s, t, near, far, 4, workers=3)
    assert np.array_equal(V, Vp)
    g = np.random.default_rng(2).standard_normal((2, m.nt)) + 0j
    q = pool.h2_solve_frequencies(m.xyz, m.tri, s, t, near, far, 4, g, workers=2)
    for k in range(2):
        assert np.allclose(V[k] @ q[k], g[k], rtol=0, atol=1e-12 * np.abs(g[k]).max())
