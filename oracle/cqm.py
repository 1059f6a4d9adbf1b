"""CQM frequencies and the R-scaled discrete Fourier transforms (Sec. 3.1).

* eq. cqm_freq: s_l = chi(R zeta^l) / dt with zeta = exp(2 pi i / L).
* eq. omega_n:  omega_n = R^{-n} / L  sum_l fhat(s_l) zeta^{-n l}.

Readings: L = N + 1 samples (the paper mixes N and N+1); chi of BDF-k is
sum_{j=1..k} (1 - z)^j / j (the paper does not write it); R defaults to
(1e-10)^{1/(2L)} so that R^L = 1e-5.  Data of the time steps are taken to the
frequencies by ghat_l = sum_n R^n b_n zeta^{n l} (the generating function of
b_n sampled on the circle of radius R), the transform whose inverse is
eq. omega_n.  Both sums are written out as plain O(L^2) products.
"""
from __future__ import annotations

import numpy as np


def default_R(N: int) -> float:
    L = N + 1
    return float((1e-10) ** (1.0 / (2.0 * L)))


def chi_bdf(z, order: int):
    """Characteristic function of the BDF method of the given order (1 or 2)."""
    if order not in (1, 2):
        raise ValueError("bdf order must be 1 or 2")
    z = np.asarray(z, dtype=np.complex128)
    out = np.zeros_like(z)
    for j in range(1, order + 1):
        out = out + (1.0 - z) ** j / j
    return out


def _zeta_pow(k, L):
    """zeta^k for integer k, reduced modulo L before the trigonometric call."""
    k = np.mod(np.asarray(k, dtype=np.int64), L)
    return np.exp(2j * np.pi * k / L)


def frequencies(N: int, dt: float, order: int, R: float | None = None):
    """The L = N + 1 CQM frequencies s_l, l = 0..N (eq. cqm_freq)."""
    if R is None:
        R = default_R(N)
    L = N + 1
    ell = np.arange(L)
    return chi_bdf(R * _zeta_pow(ell, L), order) / dt


def forward(b, R: float):
    """ghat[l] = sum_{n=0}^{N} R^n b[n] zeta^{n l}, l = 0..L-1 (b: (L, ...) real or complex)."""
    b = np.asarray(b)
    L = b.shape[0]
    n = np.arange(L)
    F = _zeta_pow(np.outer(n, n), L) * (R ** n)[None, :]     # F[l, n]
    return np.tensordot(F, b, axes=(1, 0))


def inverse(qhat, R: float):
    """q[n] = R^{-n} / L sum_{l=0}^{L-1} qhat[l] zeta^{-n l}, n = 0..L-1 (eq. omega_n)."""
    qhat = np.asarray(qhat)
    L = qhat.shape[0]
    n = np.arange(L)
    G = _zeta_pow(-np.outer(n, n), L) * (R ** (-n.astype(np.float64)) / L)[:, None]   # G[n, l]
    return np.tensordot(G, qhat, axes=(1, 0))


def weights(fhat, N: int, dt: float, order: int, R: float | None = None):
    """CQM weights omega_0..omega_N of a transfer function fhat (eq. omega_n)."""
    if R is None:
        R = default_R(N)
    s = frequencies(N, dt, order, R)
    return inverse(fhat(s), R)


def n_solved(L: int) -> int:
    """Frequencies solved under conjugate symmetry: floor(L/2) + 1."""
    return L // 2 + 1
