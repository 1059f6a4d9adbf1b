"""The double layer and the direct Dirichlet formulation on the GPU
(cqm_bem_apply_double_layer, cqm_bem_solve_dirichlet) against the oracle
(Sec. 2.2, Sec. 7.2 eq. cqmdir decoupled in frequency):

* K_l x_l equals the oracle's H^2-expanded double layer (Galerkin near
  field, far blocks U_r S_b W_c^T with the same tree and interpolation, no
  frequency compression) element by element, 1280 triangles;
* the Neumann data of a Dirichlet problem equal the oracle's (LU of the
  H^2-expanded V_l with the H^2-expanded K_l right-hand sides) in the time
  domain, 320 triangles;
* they converge to the exact Neumann data of a spherical wave from an
  interior source as the oracle's do.
"""
import numpy as np
import pytest

from oracle import cluster, cqm, dense, dlayer, pool
from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

X0 = np.array([0.1, -0.2, 0.15])


def test_apply_equals_h2_expanded_oracle():
    from paper_2006_05186_gb300 import CqmBem, build
    build.build()
    m = synth.icosphere(3)
    N, dt = 8, 0.1
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", eta=1.0, cheb_m=4, n_min=32, aca_eps=1e-13,
                rank_cap=64)
    rng = np.random.default_rng(20060518)
    x = rng.standard_normal((op.Ls, op.M)) + 1j * rng.standard_normal((op.Ls, op.M))
    y = op.apply_double_layer(x)
    op.close()
    t = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t, 1.0)
    s = cqm.frequencies(N, dt, 2)[:op.Ls]
    K = dlayer.h2_dl_matrices(m.xyz, m.tri, s, t, near, far, 4)
    ref = np.einsum("lij,lj->li", K, x)
    err = np.max(np.abs(y - ref), axis=1) / np.max(np.abs(ref), axis=1)
    print("double layer apply vs oracle per frequency:", err)
    assert np.max(err) <= 1e-10, err


def _dirichlet_gpu(level, dt, N, eps):
    from paper_2006_05186_gb300 import CqmBem, build
    build.build()
    m = synth.icosphere(level)
    g, qex = dlayer.point_source(m.xyz, m.tri, N, dt, X0, 0.6, 2.5)
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", eta=1.0, cheb_m=4, n_min=32, aca_eps=eps,
                rank_cap=64)
    q = op.solve_dirichlet(g)
    info = dict(op.last_solve_info)
    op.close()
    return m, g, qex, q, info


def test_dirichlet_equals_oracle():
    N, dt = 24, 0.2
    m, g, qex, q, info = _dirichlet_gpu(2, dt, N, 1e-12)
    assert info["converged"] == N // 2 + 1 and info["max_rel_residual"] <= 1e-13
    t = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t, 1.0)
    Ls = cqm.n_solved(N + 1)
    s = cqm.frequencies(N, dt, 2)[:Ls]
    V = pool.h2_matrices(m.xyz, m.tri, s, t, near, far, 4, workers=8)
    K = dlayer.h2_dl_matrices(m.xyz, m.tri, s, t, near, far, 4)
    q_ref, _ = dlayer.solve_dirichlet(m.xyz, m.tri, N, dt, 2, g, V=V, K=K)
    err = dense.rel_err(q, q_ref)
    print(f"Dirichlet Neumann data vs oracle: {err:.3e}")
    assert err <= 1e-6, err


def test_dirichlet_converges_to_the_spherical_wave():
    _, _, qex, q, _ = _dirichlet_gpu(2, 0.1, 48, 1e-10)
    err = np.max(np.linalg.norm(q - qex, axis=1)) / np.max(np.linalg.norm(qex, axis=1))
    print(f"Dirichlet Neumann data vs exact: {err:.3e}")
    assert err < 0.035, err
