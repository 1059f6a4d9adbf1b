"""Marching on in time on the GPU (cqm_bem_solve_mot, cqm_bem_mot_weight)
against the oracle's marching on in time (Sec. 3.2 time stepping, eq. dft)
with the H^2-expanded matrices (same tree, partition and interpolation, no
frequency compression).

* The compressed weights Vhat_n (eq. fastdft: the MACA fibres transformed,
  the slices kept) equal the oracle's weights R^-n / L sum_l V_l zeta^{-nl}
  element by element, 320-triangle sphere, N = 32, MACA tolerance 1e-12.
* The densities of the march equal the oracle's march on the 1280-triangle
  sphere (N = 64, MACA 1e-10) to 1e-6 (max over steps of the step error over
  the largest step norm), and differ from the GPU's decoupled solve by the
  O(R^L) aliasing of the latter only.
* The march is exactly causal: data that vanish up to a step give densities
  that are exactly zero up to it.
"""
import numpy as np
import pytest

from oracle import cluster, cqm, dense, incident, mot, pool
from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _h2_builder(m):
    t = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t, 1.0)
    return lambda s: pool.h2_matrices(m.xyz, m.tri, s, t, near, far, 4, workers=8)


def test_weights_equal_the_oracle():
    from paper_2006_05186_gb300 import CqmBem, build
    build.build()
    m = synth.icosphere(2)
    N, dt = 32, 0.1
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", eta=1.0, cheb_m=4, n_min=32, aca_eps=1e-12,
                rank_cap=64)
    W = {n: op.mot_weight(n) for n in (0, 1, 7, N // 2, N)}
    op.close()
    s = cqm.frequencies(N, dt, 2)
    Wref, imag_rel = mot.convolution_weights(_h2_builder(m)(s), cqm.default_R(N))
    assert imag_rel < 1e-9
    scale = np.max(np.abs(Wref[0]))
    for n, w in W.items():
        err = np.max(np.abs(w - Wref[n])) / scale
        print(f"Vhat_{n}: max |W - W_ref| / max |W_ref_0| = {err:.2e} (max |W_ref_n| / scale "
              f"{np.max(np.abs(Wref[n])) / scale:.2e})")
        assert err <= 1e-9, (n, err)
    # Vhat_0 is symmetric (canonical pair order, mirrored blocks)
    assert np.max(np.abs(W[0] - W[0].T)) <= 1e-12 * scale


@pytest.fixture(scope="module")
def sphere1280():
    from paper_2006_05186_gb300 import CqmBem, build
    build.build()
    m = synth.icosphere(3)
    N, dt = 64, 0.1
    p = synth.plane_wave_pulse()
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", eta=1.0, cheb_m=4, n_min=32, aca_eps=1e-10,
                rank_cap=64)
    b = op.rhs_plane_wave(p.direction, p.width, p.delay)
    q_mot = op.solve_mot(b)
    info = dict(op.last_solve_info)
    q_dec = op.solve(b)
    n0 = 20
    b0 = b.copy()
    b0[:n0] = 0.0
    q_causal = op.solve_mot(b0)
    op.close()
    return dict(m=m, N=N, dt=dt, b=b, q_mot=q_mot, q_dec=q_dec, info=info, n0=n0, q_causal=q_causal)


def test_march_equals_the_oracle_march(sphere1280):
    d = sphere1280
    m, N, dt = d["m"], d["N"], d["dt"]
    b_ref = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, *_pulse_args())
    assert np.max(np.abs(d["b"] - b_ref)) <= 1e-14 * np.max(np.abs(b_ref))
    q_ref, _ = mot.solve_matrices(_h2_builder(m), N, dt, 2, b_ref)
    err = dense.rel_err(d["q_mot"], q_ref)
    steps = np.linalg.norm(d["q_mot"] - q_ref, axis=1) / np.max(np.linalg.norm(q_ref, axis=1))
    print(f"march vs oracle march: {err:.3e} (worst step {int(np.argmax(steps))}); "
          f"march {d['info']['t_gmres_ms']:.1f} ms, weights {d['info']['t_forward_ms']:.1f} ms")
    assert err <= 1e-6, err
    assert d["info"]["iterations"] == N + 1


def test_march_and_decoupled_solve_differ_by_aliasing(sphere1280):
    d = sphere1280
    R = cqm.default_R(d["N"])
    diff = dense.rel_err(d["q_dec"], d["q_mot"])
    print(f"decoupled vs march: {diff:.3e} (R^L = {R ** (d['N'] + 1):.1e})")
    assert diff <= 100.0 * R ** (d["N"] + 1)


def test_march_is_exactly_causal(sphere1280):
    d = sphere1280
    q = d["q_causal"]
    assert np.all(q[:d["n0"]] == 0.0)
    assert np.max(np.abs(q[d["n0"]:])) > 0.0


def _pulse_args():
    p = synth.plane_wave_pulse()
    return p.direction, p.width, p.delay
