"""Galerkin right-hand side of an incident plane-wave pulse (Sec. 3.2, Sec. 7.2).

Reading: the single-layer problem V phi = u_inc on Gamma is solved (the paper's
sound-soft example uses the direct form with the double layer, which is not
part of this path).  For P0 test functions the L^2 projection of the data,
multiplied by the mass matrix, is the element integral:
b_n[i] = int_{tau_i} u_inc(x, t_n) dS with t_n = n dt, evaluated with Radon's
7-point rule.  The pulse is u_inc(x, t) = exp(-((t - delay - d.x) / width)^2).
"""
from __future__ import annotations

import numpy as np

from . import quadrature as Q
from .galerkin import element_geometry


def rhs_plane_wave(xyz, tri, N: int, dt: float, direction, width: float, delay: float):
    """b[n, i] for n = 0..N, i = 0..M-1 (float64, shape (N+1, M))."""
    P, area, _, _ = element_geometry(xyz, tri)
    X = np.einsum("qa,pad->pqd", Q.RADON7_BARY, P)          # (M, 7, 3)
    d = np.asarray(direction, dtype=np.float64)
    proj = X @ d                                              # (M, 7)
    t = dt * np.arange(N + 1)
    arg = (t[:, None, None] - delay - proj[None, :, :]) / width
    u = np.exp(-arg * arg)
    return np.einsum("q,nmq->nm", Q.RADON7_W, u) * area[None, :]
