"""Galerkin matrices with P1 functions for mixed boundary conditions on the
GPU (cqm_bem_p1_matrices: K with P1 trial functions, the adjoint double
layer K', the hypersingular operator D in Maue's form; Sec. 2.3 eq.
wavegalform, Sec. 3.2) against the oracle (oracle/mixed.py, pinned to the
sphere closed forms and a spherical wave), entry by entry at every solved
frequency, through host and device memory.
"""
import numpy as np
import pytest

from oracle import cqm, mixed
from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("level,N,dt", [(1, 24, 0.2), (2, 8, 0.1)])
def test_p1_matrices_equal_oracle(level, N, dt):
    from paper_2006_05186_gb300 import CqmBem, build
    build.build()
    m = synth.icosphere(level)
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", eta=1.0, cheb_m=4, n_min=32, aca_eps=1e-6)
    host = op.p1_matrices()
    dev = [t.cpu().numpy() for t in op.p1_matrices(device=True)]
    Ls = op.Ls
    op.close()
    s = cqm.frequencies(N, dt, 2)[:Ls]
    ref = mixed.p1_matrices(m.xyz, m.tri, s)
    for name, a, b, r in zip(("K1", "Kp", "D"), host, dev, ref):
        err = _rel(a, r)
        print(f"level {level}: {name} vs oracle {err:.2e}")
        assert err < 1e-10, (name, err)
        assert _rel(b, a) < 1e-13, name    # the device-memory outputs are the same sums


def test_mixed_solve_equals_oracle():
    """The mixed solve on the GPU (dense mode) equals the oracle's on the
    spherical wave of the oracle's convergence test: Dirichlet data on the
    upper, Neumann data on the lower half of the 80-triangle sphere."""
    from oracle import dlayer, galerkin
    from paper_2006_05186_gb300 import CqmBem, build
    build.build()
    m = synth.icosphere(1)
    N, dt = 24, 0.2
    x0 = np.array([0.1, -0.2, 0.15])
    _, _, cen, _ = galerkin.element_geometry(m.xyz, m.tri)
    dmask = cen[:, 2] > 0.0
    _, qn = dlayer.point_source(m.xyz, m.tri, N, dt, x0, 0.6, 2.5)
    uv = mixed.point_source_vertices(m.xyz, N, dt, x0, 0.6, 2.5)
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="dense")
    q, u = op.solve_mixed(dmask, uv, qn)
    op.close()
    q_ref, u_ref, info = mixed.solve_mixed(m.xyz, m.tri, N, dt, 2, dmask, uv, qn)
    ED, VN = info["ED"], info["VN"]
    eq, eu = _rel(q[:, ED], q_ref), _rel(u[:, VN], u_ref)
    print(f"mixed solve vs oracle: q {eq:.2e}, u {eu:.2e}")
    assert eq < 1e-8 and eu < 1e-8, (eq, eu)
    # outside their parts the results are zero
    assert np.all(q[:, ~dmask] == 0.0) and np.count_nonzero(u) <= u.shape[0] * len(VN)
