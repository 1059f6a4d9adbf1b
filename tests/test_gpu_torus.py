"""The torus workload (major radius 1, minor radius 0.3; Sec. 7 uses closed
surfaces of this kind), reduced to a size the oracle solves in full: 1280
triangles (n_u = 40, n_v = 16), BDF2, N = 128, dt = 0.4 times the mean edge
length (Courant number 0.4), MACA tolerance 1e-9, all other parameters at
their defaults (bf16 tensor-core far coupling and FP32 near field in the inner
iterations, float-float residuals).

The oracle solves the same problem from scratch at all 65 solved frequencies
(LU of its H^2-expanded V_l) and transforms back; the time-domain densities
must agree to 1e-6 at every step.  The full 20480-triangle, N = 1024 torus
is measured by the benchmark against the same path at MACA 1e-11.
"""
import numpy as np
import pytest

from oracle import cluster, cqm, dense, incident, pool
from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_reduced_torus_time_domain_vs_oracle():
    from paper_2006_05186_gb300 import CqmBem, build
    build.build()
    m = synth.torus_for(1280)
    N = 128
    dt = 0.4 * synth.mean_edge_length(m)
    p = synth.plane_wave_pulse()
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", aca_eps=1e-9)
    assert op.info()["n_far"] > 0
    b = op.rhs_plane_wave(p.direction, p.width, p.delay)
    q = op.solve(b)
    info = op.last_solve_info
    op.close()
    assert info["converged"] == op.Ls and info["max_rel_residual"] <= 1e-13
    L = N + 1
    R = cqm.default_R(N)
    t = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t, 1.0)
    b_ref = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, p.delay)
    assert np.max(np.abs(b - b_ref)) <= 1e-14 * np.max(np.abs(b_ref))
    g = cqm.forward(b_ref, R)
    s = cqm.frequencies(N, dt, 2)
    Ls = L // 2 + 1
    qh = pool.h2_solve_frequencies(m.xyz, m.tri, s[:Ls], t, near, far, 4, g[:Ls])
    q_ref = cqm.inverse(dense.fill_conjugate(qh, L), R).real
    err = dense.rel_err(q, q_ref)
    print(f"reduced torus: time-domain rel err vs the oracle {err:.3e}")
    assert err <= 1e-6, err
