"""Pins of the mixed-boundary-condition oracle (Sec. 2.3 eq. wavegalform,
Sec. 3.2 eq. cqmgalapx, decoupled in frequency): P1 trial and test functions,
the adjoint double layer K' and the hypersingular operator D in Maue's form,
against what the mathematics fixes:

* the P1 hats sum to one, so K with P1 trial functions applied to the vertex
  vector of ones is the P0 double layer applied to ones (pinned by Gauss's
  identity and the sphere closed form in test_oracle_dlayer);
* K' is the transpose of K (test and trial roles exchanged) and D is
  symmetric, both up to the quadrature's asymmetry;
* the unit sphere: on the restriction of x_3 (a degree-one spherical
  harmonic) and on constants, K and D act by their closed-form eigenvalues
  K Y_n = (1/2 + s^2 i_n k_n') Y_n and D Y_n = -s^3 i_n' k_n' Y_n (modified
  spherical Bessel functions), O(h^2) with refinement, and at s = 0 by the
  Laplace values -1/6 and 2/3, D 1 = 0 exactly;
* a spherical wave from a source inside the sphere with Dirichlet data on the
  upper and Neumann data on the lower half: the unknown Neumann and Dirichlet
  data converge to the exact traces, and flipping the sign of K' or of D (a
  plausible mistake) does not;
* the paper's own time stepping of the mixed system (eqs. cqmgalapx and
  cqmrhs) is exactly causal and agrees with the decoupled solve to R^L.
"""
import numpy as np
import pytest

from oracle import cqm, dlayer, galerkin, mixed
from paper_2006_05186_gb300 import synth

X0 = np.array([0.1, -0.2, 0.15])
S = np.array([1.0, 3.0 + 2.0j])


@pytest.fixture(scope="module")
def spheres():
    out = {}
    for level in (1, 2):
        m = synth.icosphere(level)
        out[level] = (m, mixed.p1_matrices(m.xyz, m.tri, np.concatenate([[0.0], S])))
    return out


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_partition_of_unity_gives_the_p0_double_layer(spheres):
    m, (K1, _, _) = spheres[1]
    K0 = dlayer.dense_dl_matrices(m.xyz, m.tri, np.concatenate([[0.0], S]))
    one_v, one_t = np.ones(len(m.xyz)), np.ones(len(m.tri))
    assert _rel(K1 @ one_v, K0 @ one_t) < 1e-12


def test_adjoint_and_symmetry(spheres):
    for level in (1, 2):
        _, (K1, Kp, D) = spheres[level]
        assert _rel(Kp, np.transpose(K1, (0, 2, 1))) < 1e-5
        assert _rel(D, np.transpose(D, (0, 2, 1))) < 1e-7


def test_closed_forms_reach_the_laplace_values():
    # K Y_0 is the double-layer closed form pinned in test_oracle_dlayer
    for s in (0.5, 2.0 + 1.0j):
        assert abs(mixed.sphere_eig_K(0, s) - (0.5 - (1 + s) * np.exp(-s) * np.sinh(s) / s)) < 1e-14
    # the classical Laplace eigenvalues as s -> 0
    assert abs(mixed.sphere_eig_K(1, 1e-3) + 1.0 / 6.0) < 1e-5
    assert abs(mixed.sphere_eig_D(1, 1e-3) - 2.0 / 3.0) < 1e-5
    assert abs(mixed.sphere_eig_D(0, 1e-3)) < 1e-5


def _errors(m, K1, D, k, lK1, lD1, lD0):
    Im = mixed.mass_p0p1(m.xyz, m.tri)
    M11 = mixed.mass_p1p1(m.xyz, m.tri)
    z = m.xyz[:, 2] / np.linalg.norm(m.xyz, axis=1)
    one = np.ones(len(m.xyz))
    return (_rel(K1[k] @ z, lK1 * (Im @ z)), _rel(D[k] @ z, lD1 * (M11 @ z)),
            np.max(np.abs(D[k] @ one - lD0 * (M11 @ one))) / np.max(np.abs(M11 @ one)))


def test_laplace_limit_on_the_sphere(spheres):
    errs = [_errors(spheres[lv][0], spheres[lv][1][0], spheres[lv][1][2], 0, -1.0 / 6.0, 2.0 / 3.0, 0.0)
            for lv in (1, 2)]
    (k1, d1, c1), (k2, d2, c2) = errs
    assert c1 < 1e-13 and c2 < 1e-13               # D 1 = 0: the curls of the hats sum to zero
    assert k2 < 1e-2 and k1 / k2 > 2.5, (k1, k2)
    assert d2 < 1.5e-2 and d1 / d2 > 2.5, (d1, d2)


@pytest.mark.parametrize("k", [1, 2])
def test_sphere_eigenvalues_converge(spheres, k):
    s = S[k - 1]
    lam = (mixed.sphere_eig_K(1, s), mixed.sphere_eig_D(1, s), mixed.sphere_eig_D(0, s))
    e1 = _errors(spheres[1][0], spheres[1][1][0], spheres[1][1][2], k, *lam)
    e2 = _errors(spheres[2][0], spheres[2][1][0], spheres[2][1][2], k, *lam)
    for a, b in zip(e1, e2):
        assert b < 2e-2 and a / b > 2.0, (e1, e2)


def _mixed_error(level, dt, N, flip=None):
    m = synth.icosphere(level)
    _, _, cen, _ = galerkin.element_geometry(m.xyz, m.tri)
    dmask = cen[:, 2] > 0.0
    _, qn = dlayer.point_source(m.xyz, m.tri, N, dt, X0, 0.6, 2.5)
    uv = mixed.point_source_vertices(m.xyz, N, dt, X0, 0.6, 2.5)
    Ls = cqm.n_solved(N + 1)
    s = cqm.frequencies(N, dt, 2)[:Ls]
    V = galerkin.dense_matrices(m.xyz, m.tri, s)
    K1, Kp, D = mixed.p1_matrices(m.xyz, m.tri, s)
    out = {}
    for f in [None] + list(flip or []):
        mats = (V, K1, -Kp if f == "Kp" else Kp, -D if f == "D" else D)
        q, u, info = mixed.solve_mixed(m.xyz, m.tri, N, dt, 2, dmask, uv, qn, mats=mats)
        assert info["max_imag"] < 1e-10
        ED, VN = info["ED"], info["VN"]
        eq = np.max(np.linalg.norm(q - qn[:, ED], axis=1)) / np.max(np.linalg.norm(qn[:, ED], axis=1))
        eu = np.max(np.linalg.norm(u - uv[:, VN], axis=1)) / np.max(np.linalg.norm(uv[:, VN], axis=1))
        out[f] = (eq, eu)
    return out


def test_mixed_spherical_wave_converges():
    e1 = _mixed_error(1, 0.2, 24, flip=["Kp", "D"])
    e2 = _mixed_error(2, 0.1, 48)
    (q1, u1), (q2, u2) = e1[None], e2[None]
    assert q2 < 0.05 and u2 < 0.03, e2
    assert q1 / q2 > 3.0 and u1 / u2 > 3.0, (e1, e2)
    # a sign error in K' or in D leaves the solution far from the traces
    assert e1["Kp"][1] > 1.0 and e1["D"][1] > 1.0, e1


def test_marching_on_in_time_agrees_with_the_decoupled_solve():
    """The paper's own time stepping of the mixed system (eqs. cqmgalapx and
    cqmrhs, the weights of eq. dft) is exactly causal and agrees with the
    decoupled frequency-domain solve to the order R^L of the wrap-around."""
    m = synth.icosphere(1)
    N, dt = 24, 0.2
    _, _, cen, _ = galerkin.element_geometry(m.xyz, m.tri)
    dmask = cen[:, 2] > 0.0
    _, qn = dlayer.point_source(m.xyz, m.tri, N, dt, X0, 0.6, 2.5)
    uv = mixed.point_source_vertices(m.xyz, N, dt, X0, 0.6, 2.5)
    s = cqm.frequencies(N, dt, 2)
    mats = (galerkin.dense_matrices(m.xyz, m.tri, s),) + mixed.p1_matrices(m.xyz, m.tri, s)
    Ls = cqm.n_solved(N + 1)
    qd, ud, _ = mixed.solve_mixed(m.xyz, m.tri, N, dt, 2, dmask, uv, qn, mats=[a[:Ls] for a in mats])
    qm, um, info = mixed.solve_mixed_mot(m.xyz, m.tri, N, dt, 2, dmask, uv, qn, mats_all=mats)
    RL = cqm.default_R(N) ** (N + 1)
    assert info["imag_rel"] < 1e-9
    assert _rel(qm, qd) < RL and _rel(um, ud) < RL, (_rel(qm, qd), _rel(um, ud))
    # causality: data from step 10 on do not change the first ten steps
    qn2, uv2 = qn.copy(), uv.copy()
    qn2[10:] *= 2.0
    uv2[10:] += 1.0
    qm2, um2, _ = mixed.solve_mixed_mot(m.xyz, m.tri, N, dt, 2, dmask, uv2, qn2, mats_all=mats)
    assert np.array_equal(qm2[:10], qm[:10]) and np.array_equal(um2[:10], um[:10])
    assert _rel(qm2[10:], qm[10:]) > 0.1


def test_h2_p1_operators_converge_with_m():
    """The H^2 form of the P1 operators (Sec. 4: far blocks of triangle
    clusters through the interpolated kernel, with the P1 double-layer, curl
    and normal bases) converges to the Galerkin matrices as the number m of
    Chebyshev points per axis grows; its hats still sum to one (the P1 double
    layer on ones is the H^2 P0 double layer on ones), its far blocks keep
    K' = K^T and the symmetry of D exactly."""
    from oracle import cluster
    m = synth.icosphere(2)
    t = cluster.build_tree(m.xyz, m.tri, 16)
    near, far = cluster.partition(t, 1.0)
    assert len(far) > 0
    s = np.array([1.5, 3.0 + 2.0j])
    ref = mixed.p1_matrices(m.xyz, m.tri, s)
    errs = []
    for mm in (2, 3, 4):
        h = mixed.h2_p1_matrices(m.xyz, m.tri, s, t, near, far, mm)
        errs.append([_rel(a, b) for a, b in zip(h, ref)])
    errs = np.array(errs)                        # (m, operator)
    assert np.all(errs[1] < errs[0] / 3.0) and np.all(errs[2] < errs[1] / 3.0), errs
    assert errs[2][0] < 1e-3 and errs[2][2] < 1e-5, errs
    K1h, Kph, Dh = h
    K0h = dlayer.h2_dl_matrices(m.xyz, m.tri, s, t, near, far, 4)
    assert _rel(K1h @ np.ones(len(m.xyz)), K0h @ np.ones(len(m.tri))) < 1e-12
    assert _rel(Kph, np.transpose(K1h, (0, 2, 1))) < 1e-5
    assert _rel(Dh, np.transpose(Dh, (0, 2, 1))) < 1e-7
