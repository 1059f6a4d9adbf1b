"""Pins of the CQM frequencies and R-scaled transforms (Sec. 3.1, eqs. omega_n,
cqm_freq) against closed-form CQM weights of known transfer functions."""
import math

import numpy as np
import pytest

from oracle import cqm


def aliased(w_fn, n, L, R, terms=8):
    """The L-point R-scaled transform returns sum_j omega_{n+jL} R^{jL}."""
    return sum(w_fn(n + j * L) * R ** (j * L) for j in range(terms))


@pytest.mark.parametrize("N", [32, 256])
def test_T1_bdf1_inverse_s(N):
    dt = 0.1
    R = cqm.default_R(N)
    L = N + 1
    w = cqm.weights(lambda s: 1.0 / s, N, dt, 1, R)
    ref = dt / (1.0 - R ** L)
    assert np.max(np.abs(w - ref)) / dt < 1e-10


@pytest.mark.parametrize("N", [32, 256])
def test_T1_bdf2_inverse_s(N):
    dt = 0.1
    R = cqm.default_R(N)
    L = N + 1
    w = cqm.weights(lambda s: 1.0 / s, N, dt, 2, R)
    n = np.arange(L)
    ref = dt * (1.0 / (1.0 - R ** L) - 3.0 ** (-(n + 1.0)) / (1.0 - (R / 3.0) ** L))
    assert np.max(np.abs(w - ref)) / dt < 1e-10


def test_T2_bdf1_kernel_poisson():
    N, dt, r = 32, 0.1, 0.37
    R = cqm.default_R(N)
    lam = r / dt
    w = cqm.weights(lambda s: np.exp(-s * r), N, dt, 1, R)
    pois = lambda n: math.exp(-lam + n * math.log(lam) - math.lgamma(n + 1))
    ref = np.array([aliased(pois, n, N + 1, R, terms=3) for n in range(N + 1)])
    assert np.max(np.abs(w - ref)) < 1e-10


def _hermite(n, x):
    h0, h1 = 1.0, 2.0 * x
    if n == 0:
        return h0
    for k in range(1, n):
        h0, h1 = h1, 2.0 * x * h1 - 2.0 * k * h0
    return h1


def test_T2_bdf2_kernel_hermite():
    N, dt, r = 32, 0.1, 0.37
    R = cqm.default_R(N)
    lam = r / dt
    w = cqm.weights(lambda s: np.exp(-s * r), N, dt, 2, R)
    x = math.sqrt(2.0 * lam)
    wn = lambda n: (math.exp(-1.5 * lam + (n / 2.0) * math.log(lam / 2.0) - math.lgamma(n + 1))
                    * _hermite(n, x))
    ref = np.array([aliased(wn, n, N + 1, R, terms=2) for n in range(N + 1)])
    assert np.max(np.abs(w - ref)) < 1e-10


def test_frequencies_values_and_symmetry():
    N, dt = 32, 0.1
    s = cqm.frequencies(N, dt, 2)
    R = cqm.default_R(N)
    assert abs(R - 0.70548) < 1e-5
    assert abs(R ** (N + 1) - 1e-5) < 1e-15
    assert abs(s[0].imag) < 1e-14 and abs(s[0].real - 3.3792) < 1e-3
    # chi(-R)/dt is the largest modulus: (1+R) + (1+R)^2/2
    assert abs(np.max(np.abs(s)) - ((1 + R) + (1 + R) ** 2 / 2) / dt) < 0.3
    L = N + 1
    for l in range(1, L):
        assert abs(s[L - l] - np.conj(s[l])) < 1e-12
    assert np.all(s.real > 0)


@pytest.mark.parametrize("N", [32, 256, 1024])
def test_T10_round_trip_and_conjugate_symmetry(N):
    rng = np.random.default_rng(7)
    L = N + 1
    R = cqm.default_R(N)
    b = rng.standard_normal((L, 3))
    g = cqm.forward(b, R)
    for l in range(1, L):
        assert np.allclose(g[L - l], np.conj(g[l]), atol=1e-12 * np.abs(g).max())
    back = cqm.inverse(g, R)
    floor = 1e-16 * R ** (-N) * L
    assert np.max(np.abs(back - b)) < 10 * floor
    assert np.max(np.abs(back.imag)) < 10 * floor


def test_planted_sign_error_is_caught(monkeypatch):
    """A transform with the wrong exponent sign fails the BDF2 pin."""
    N, dt = 32, 0.1
    good = cqm._zeta_pow
    monkeypatch.setattr(cqm, "_zeta_pow", lambda k, L: np.conj(good(k, L)))
    R = cqm.default_R(N)
    L = N + 1
    w = cqm.inverse(1.0 / cqm.frequencies(N, dt, 2, R) + 0j, R)
    n = np.arange(L)
    ref = dt * (1.0 / (1.0 - R ** L) - 3.0 ** (-(n + 1.0)) / (1.0 - (R / 3.0) ** L))
    # with both signs flipped the frequencies flip too; weights of a real
    # transfer function are unchanged -- flip only the inverse to plant a bug
    monkeypatch.setattr(cqm, "_zeta_pow", good)
    s = cqm.frequencies(N, dt, 2, R)
    monkeypatch.setattr(cqm, "_zeta_pow", lambda k, L: np.conj(good(k, L)))
    w_bad = cqm.inverse(1.0 / s, R)
    assert np.max(np.abs(w_bad - ref)) / dt > 1e-3
