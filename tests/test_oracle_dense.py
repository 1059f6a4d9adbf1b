"""Pins of the whole frequency-domain pipeline (Remark in Sec. 6.2):
conjugate symmetry, causality, and the scalar CQM limit on the sphere."""
import numpy as np

from oracle import cqm, dense, galerkin as G, incident
from paper_2006_05186_gb300 import synth


def test_conjugate_symmetry_all_frequencies():
    m = synth.icosphere(0)
    N, dt = 12, 0.1
    p = synth.plane_wave_pulse(width=0.5)
    b = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, p.delay - 2.0)
    q_all, info = dense.solve(m.xyz, m.tri, N, dt, 2, b, all_frequencies=True)
    q_half, info2 = dense.solve(m.xyz, m.tri, N, dt, 2, b)
    L = N + 1
    qh = info["qhat"]
    for l in range(1, L):
        assert np.allclose(qh[L - l], np.conj(qh[l]), rtol=0, atol=1e-12 * np.abs(qh).max())
    assert info["max_imag"] < 1e-8 * np.abs(q_all).max()
    assert dense.rel_err(q_half, q_all) < 1e-10


def test_causality_late_data():
    """b_n = 0 for n < n0 gives q_n = O(R^L) for n < n0 (circular wrap-around)."""
    m = synth.icosphere(0)
    N, dt, n0 = 16, 0.1, 8
    rng = np.random.default_rng(3)
    b = np.zeros((N + 1, m.nt))
    b[n0:] = rng.standard_normal((N + 1 - n0, m.nt))
    q, _ = dense.solve(m.xyz, m.tri, N, dt, 2, b)
    R = cqm.default_R(N)
    assert np.max(np.abs(q[:n0])) < 100 * R ** (N + 1) * np.max(np.abs(q))
    assert np.max(np.abs(q[n0:])) > 1e-3 * np.max(np.abs(q))


def test_T4_scalar_limit_on_sphere():
    """Data constant over the sphere: the mesh solution tends to the scalar CQM
    with transfer function 1/lambda_0(s) as the mesh is refined."""
    N, dt, bdf = 8, 0.25, 2
    R = cqm.default_R(N)
    t = dt * np.arange(N + 1)
    g = np.exp(-((t - 1.2) / 0.5) ** 2)
    s = cqm.frequencies(N, dt, bdf, R)
    lam0 = (1.0 - np.exp(-2.0 * s)) / (2.0 * s)
    q_scalar = cqm.inverse(cqm.forward(g, R) / lam0, R).real
    errs = []
    for lev in (0, 1, 2):
        m = synth.icosphere(lev)
        _, area, _, _ = G.element_geometry(m.xyz, m.tri)
        b = g[:, None] * area[None, :]
        q, _ = dense.solve(m.xyz, m.tri, N, dt, bdf, b)
        qmean = (q @ area) / np.sum(area)
        errs.append(np.max(np.abs(qmean - q_scalar)) / np.max(np.abs(q_scalar)))
    assert errs[2] < errs[1] < errs[0], errs
    assert errs[2] < 0.02, errs


def test_rhs_plane_wave_smooth_data():
    """Incident pulse data: zero initial data to e^-16, peak value |tau| at the arrival."""
    m = synth.icosphere(2)
    p = synth.plane_wave_pulse()
    N, dt = 32, 0.1
    b = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, p.delay)
    _, area, _, _ = G.element_geometry(m.xyz, m.tri)
    assert np.all(np.abs(b[0]) <= np.exp(-16) * area * 1.0001)
    assert np.all(b <= area[None, :] * (1 + 1e-12))
    assert np.max(b / area[None, :]) > 0.5


def _arrival_steps(b, dt):
    """Peak time of each element's data b_n[i], refined by the parabola through
    the largest sample and its two neighbours."""
    n = np.argmax(b, axis=0)
    n = np.clip(n, 1, b.shape[0] - 2)
    i = np.arange(b.shape[1])
    y0, y1, y2 = b[n - 1, i], b[n, i], b[n + 1, i]
    return (n + 0.5 * (y0 - y2) / (y0 - 2.0 * y1 + y2)) * dt


def test_rhs_plane_wave_arrival_follows_direction():
    """The pulse u(x, t) = exp(-((t - delay - d.x)/w)^2) reaches x at
    t = delay + d.x: each element's data peaks at delay + d.c_i (c_i the
    centroid; the 7-point rule integrates the linear d.x exactly, and the
    pulse is wide against the element), so for d = +z the elements at z = -1
    peak 2/dt steps before those at z = +1.  Reversing the sign of d.x in the
    oracle (planted here as the opposite direction) fails the check."""
    m = synth.icosphere(2)
    p = synth.plane_wave_pulse(width=0.5)
    N, dt = 300, 0.02
    _, _, cen, _ = G.element_geometry(m.xyz, m.tri)
    expect = p.delay + cen @ p.direction
    for d, ok in ((p.direction, True), (-p.direction, False)):
        b = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, d, p.width, p.delay)
        t_peak = _arrival_steps(b, dt)
        err = np.max(np.abs(t_peak - expect))
        # element size (h ~ 0.2) and the sampling refine to well below dt
        assert (err < 0.25 * dt) == ok, (ok, err)
    b = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, p.delay)
    t_peak = _arrival_steps(b, dt)
    south, north = cen[:, 2] < -0.9, cen[:, 2] > 0.9
    lead = np.mean(t_peak[north]) - np.mean(t_peak[south])
    assert abs(lead - (np.mean(cen[north, 2]) - np.mean(cen[south, 2]))) < 0.05 * dt
    assert lead > 1.8
