"""Marching-on-in-time CQM solve of the single layer (Sec. 3.2, the time
stepping of the Galerkin CQM system; Sec. 6.2, eq. dft).

Test infrastructure only (see the package docstring).

The CQM integration weights of the Galerkin single layer are the matrices

    Vhat_n = R^{-n} / L  sum_{l=0}^{L-1} V_l zeta^{-n l},   n = 0..N

(eq. dft with the L = N + 1 reading), real up to rounding because the
frequencies come in conjugate pairs.  The time-discrete system is the causal
convolution

    sum_{k=0}^{n} Vhat_{n-k} q_k = b_n,   n = 0..N,

solved step by step: Vhat_0 q_n = b_n - sum_{k<n} Vhat_{n-k} q_k, with Vhat_0
factorised once (the paper factorises it by LU; here scipy's LAPACK LU, a
library primitive).  Unlike the decoupled frequency-domain solve
(``oracle.dense``), which solves the same convolution with the wrap-around
terms weighted by R^L, this is exactly causal.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import lu_factor, lu_solve

from . import cqm
from .galerkin import QuadParams, dense_matrices


def convolution_weights(mats_all, R: float):
    """Vhat_n, n = 0..L-1, from V_l of all L frequencies (eq. dft).

    Returns (weights (L, ...) real, largest |imaginary part| relative to the
    largest |weight|)."""
    W = cqm.inverse(np.asarray(mats_all), R)
    scale = float(np.max(np.abs(W))) or 1.0
    return W.real.copy(), float(np.max(np.abs(W.imag))) / scale


def solve_matrices(build, N: int, dt: float, bdf: int, rhs, R: float | None = None):
    """Densities q_n (N+1, M) for data b_n (N+1, M) by marching on in time.

    `build(s)` returns the stack V_l (len(s), M, M) for the frequencies s.
    Returns (q, info) with info = {weights, imag_rel}."""
    if R is None:
        R = cqm.default_R(N)
    L = N + 1
    b = np.asarray(rhs, dtype=np.float64)
    s = cqm.frequencies(N, dt, bdf, R)
    W, imag_rel = convolution_weights(build(s), R)
    lu = lu_factor(W[0])
    q = np.zeros_like(b)
    for n in range(L):
        f = b[n].copy()
        for k in range(n):
            f -= W[n - k] @ q[k]
        q[n] = lu_solve(lu, f)
    return q, {"weights": W, "imag_rel": imag_rel}


def solve(xyz, tri, N: int, dt: float, bdf: int, rhs, R: float | None = None,
          qp: QuadParams = QuadParams()):
    """Marching-on-in-time solve with the dense Galerkin matrices V_l (Sec. 3.2)."""
    return solve_matrices(lambda ss: dense_matrices(xyz, tri, ss, qp), N, dt, bdf, rhs, R)
