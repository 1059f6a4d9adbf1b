"""Pins of the marching-on-in-time oracle (Sec. 3.2 time stepping, eq. dft).

* a scalar transfer function 1/s (integration): its CQM convolution is
  inverted by the BDF difference quotient, exactly up to the R^L aliasing of
  the weights;
* exact causality: data that vanish up to a step give a density that
  vanishes up to it, where the decoupled frequency-domain solve is only
  O(R^L) small;
* on the sphere, marching on in time and the decoupled solve agree to O(R^L);
* the weights are real (conjugate frequency pairs).
"""
import numpy as np
import pytest

from oracle import cqm, dense, incident, mot
from paper_2006_05186_gb300 import synth


def _scalar_inverse_s(s):
    return (1.0 / s).reshape(-1, 1, 1)


@pytest.mark.parametrize("bdf", [1, 2])
def test_inverse_s_is_inverted_by_the_bdf_difference_quotient(bdf):
    N, dt = 40, 0.05
    t = dt * np.arange(N + 1)
    g = (t ** 3 * np.exp(-3.0 * t))[:, None]
    q, info = mot.solve_matrices(_scalar_inverse_s, N, dt, bdf, g)
    gp = np.concatenate([[0.0, 0.0], g[:, 0]])  # g_{-1} = g_{-2} = 0
    if bdf == 1:
        ref = (gp[2:] - gp[1:-1]) / dt
    else:
        ref = (1.5 * gp[2:] - 2.0 * gp[1:-1] + 0.5 * gp[:-2]) / dt
    R = cqm.default_R(N)
    err = np.max(np.abs(q[:, 0] - ref)) / np.max(np.abs(ref))
    assert err < 5.0 * R ** (N + 1), err
    assert info["imag_rel"] < 1e-10


def test_marching_is_exactly_causal():
    m = synth.icosphere(1)
    N, dt, n0 = 16, 0.25, 5
    p = synth.plane_wave_pulse(width=0.5)
    b = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, p.delay - 2.0)
    b[:n0] = 0.0
    q, _ = mot.solve(m.xyz, m.tri, N, dt, 2, b)
    assert np.all(q[:n0] == 0.0)
    assert np.max(np.abs(q[n0:])) > 0.0
    qd, _ = dense.solve(m.xyz, m.tri, N, dt, 2, b)
    lead = np.max(np.abs(qd[:n0])) / np.max(np.abs(qd))
    assert lead <= 10.0 * cqm.default_R(N) ** (N + 1)


def test_marching_agrees_with_decoupled_solve_to_aliasing_order():
    m = synth.icosphere(1)
    N, dt = 16, 0.25
    p = synth.plane_wave_pulse(width=0.5)
    b = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, p.delay - 2.0)
    qm, info = mot.solve(m.xyz, m.tri, N, dt, 2, b)
    qd, _ = dense.solve(m.xyz, m.tri, N, dt, 2, b)
    assert dense.rel_err(qm, qd) <= cqm.default_R(N) ** (N + 1)
    assert info["imag_rel"] < 1e-10
