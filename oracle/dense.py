"""Decoupled frequency-domain CQM solve of the single layer (Remark in Sec. 6.2).

Steps, in the paper's terms:
1. ghat_l = sum_n R^n b_n zeta^{n l}               (transform of the data)
2. V_l qhat_l = ghat_l, l = 0..L-1                  (one Helmholtz system per
   frequency s_l, eq. cqm_freq, dense V_l of Sec. 3.2, complex LU)
3. q_n = R^{-n}/L sum_l qhat_l zeta^{-n l}          (eq. omega_n)
With conjugate symmetry (s_{L-l} = conj s_l, real data) only l < floor(L/2)+1
need solving; `all_frequencies=True` solves all L and is used to check that
symmetry.  The matrix solve is numpy's LAPACK LU (a library primitive).
"""
from __future__ import annotations

import numpy as np

from . import cqm
from .galerkin import QuadParams, dense_matrices


def solve_frequencies(mats, ghat):
    """qhat_l = V_l^{-1} ghat_l for a stack of matrices (L', M, M) and data (L', M)."""
    return np.stack([np.linalg.solve(mats[k], ghat[k]) for k in range(len(mats))])


def fill_conjugate(qhat_half, L):
    """Extend l < floor(L/2)+1 to all l by qhat_{L-l} = conj(qhat_l)."""
    Ls = cqm.n_solved(L)
    out = np.empty((L,) + qhat_half.shape[1:], dtype=np.complex128)
    out[:Ls] = qhat_half[:Ls]
    for l in range(Ls, L):
        out[l] = np.conj(qhat_half[L - l])
    return out


def solve(xyz, tri, N: int, dt: float, bdf: int, rhs, R: float | None = None,
          qp: QuadParams = QuadParams(), all_frequencies: bool = False,
          matrices=None):
    """Densities q_n (N+1, M) for right-hand sides b_n (N+1, M).

    `matrices(s)` may supply the V_l stack for the frequencies s (the
    H^2-expanded oracle passes its own); default: dense Galerkin matrices.
    Returns (q, info) with info = {qhat, max_imag, s}.
    """
    if R is None:
        R = cqm.default_R(N)
    L = N + 1
    s = cqm.frequencies(N, dt, bdf, R)
    ghat = cqm.forward(np.asarray(rhs, dtype=np.float64), R)
    nl = L if all_frequencies else cqm.n_solved(L)
    build = matrices if matrices is not None else (lambda ss: dense_matrices(xyz, tri, ss, qp))
    mats = build(s[:nl])
    qhat = solve_frequencies(mats, ghat[:nl])
    if not all_frequencies:
        qhat = fill_conjugate(qhat, L)
    q = cqm.inverse(qhat, R)
    return q.real.copy(), {"qhat": qhat, "max_imag": float(np.max(np.abs(q.imag))), "s": s}


def rel_err(q, q_ref):
    """max_n ||q_n - q_ref_n||_2 / max_n ||q_ref_n||_2 (time steps along axis 0)."""
    num = np.max(np.linalg.norm(np.asarray(q) - np.asarray(q_ref), axis=1))
    den = np.max(np.linalg.norm(np.asarray(q_ref), axis=1))
    return float(num / den)
