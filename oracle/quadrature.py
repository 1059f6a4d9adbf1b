"""Element quadrature rules (the paper leaves quadrature open, Sec. 3.2).

Reference triangle T^ = {(x1, x2): 0 <= x2 <= x1 <= 1} (area 1/2) with the
parametrisation chi(x^) = P0 + x1 (P1 - P0) + x2 (P2 - P1), whose Jacobian is
2|tau|.  Barycentric coordinates of chi(x^) are (1 - x1, x1 - x2, x2).

Rules:
* Radon's degree-5 seven-point rule (closed form with sqrt(15)), used for
  regular pairs (7 x 7 points).
* A collapsed (Duffy) Gauss-Legendre rule, x1 = u, x2 = u v, with g points per
  direction, used for near-singular pairs (g^2 x g^2 points).
* The Sauter-Schwab relative-coordinate rules for identical triangles (6
  regions), a common edge (5 regions) and a common vertex (2 regions), each a
  g^4 Gauss-Legendre tensor rule on [0,1]^4 (Sauter & Schwab, Boundary Element
  Methods, Springer 2011, Sec. 5.2).

Parity pins: polynomial exactness of each rule (Radon to degree 5, collapsed to
degree 2g-2, every Sauter-Schwab region set reproduces integrals of polynomials
over T^ x T^), and the singular rules against the closed-form in-plane Laplace
potential (tests/test_oracle_quadrature.py).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

_SQ15 = math.sqrt(15.0)
_A = (6.0 - _SQ15) / 21.0
_B = (6.0 + _SQ15) / 21.0

#: Radon's seven-point rule: barycentric points, weights summing to one.
RADON7_BARY = np.array([
    [1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0],
    [_A, _A, 1.0 - 2.0 * _A],
    [_A, 1.0 - 2.0 * _A, _A],
    [1.0 - 2.0 * _A, _A, _A],
    [_B, _B, 1.0 - 2.0 * _B],
    [_B, 1.0 - 2.0 * _B, _B],
    [1.0 - 2.0 * _B, _B, _B],
])
RADON7_W = np.array([9.0 / 40.0] + [(155.0 - _SQ15) / 1200.0] * 3
                    + [(155.0 + _SQ15) / 1200.0] * 3)


def gauss_legendre01(g: int):
    """Gauss-Legendre nodes and weights on [0, 1] (weights sum to 1)."""
    x, w = np.polynomial.legendre.leggauss(g)
    return (x + 1.0) / 2.0, w / 2.0


def collapsed_rule(g: int):
    """Duffy-collapsed Gauss rule on the triangle: barycentric points (g*g, 3),
    weights summing to one.  Point (a, b) -> x1 = u_a, x2 = u_a v_b."""
    x, w = gauss_legendre01(g)
    pts, wts = [], []
    for a in range(g):
        for b in range(g):
            x1 = x[a]
            x2 = x[a] * x[b]
            pts.append([1.0 - x1, x1 - x2, x2])
            wts.append(2.0 * w[a] * w[b] * x[a])
    return np.array(pts), np.array(wts)


def _grid4(g: int):
    x, w = gauss_legendre01(g)
    X = np.array(list(itertools.product(x, x, x, x)))
    W = np.prod(np.array(list(itertools.product(w, w, w, w))), axis=1)
    return X[:, 0], X[:, 1], X[:, 2], X[:, 3], W


def sauter_schwab(case: str, g: int):
    """Relative-coordinate rule on T^ x T^ for a singular pair.

    Returns (xh, yh, w): reference points of the test and trial triangle,
    shapes (n, 2), and weights (n,) summing to |T^|^2 = 1/4.  The pair
    integral is 4 |tau| |t| sum_k w_k k(chi_tau(xh_k), chi_t(yh_k)).

    case 'ident': same triangle, same parametrisation.
    case 'edge':  both parametrised with the shared edge as chi(s, 0), same
                  direction (P0, P1 shared).
    case 'vert':  both parametrised with the shared vertex as P0.
    """
    xi, e1, e2, e3, W = _grid4(g)
    if case == "ident":
        wt = xi ** 3 * e1 ** 2 * e2
        regions = [
            ((xi, xi * (1 - e1 + e1 * e2)), (xi * (1 - e1 * e2 * e3), xi * (1 - e1)), wt),
            ((xi * (1 - e1 * e2 * e3), xi * (1 - e1)), (xi, xi * (1 - e1 + e1 * e2)), wt),
            ((xi, xi * e1 * (1 - e2 + e2 * e3)), (xi * (1 - e1 * e2), xi * e1 * (1 - e2)), wt),
            ((xi * (1 - e1 * e2), xi * e1 * (1 - e2)), (xi, xi * e1 * (1 - e2 + e2 * e3)), wt),
            ((xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), (xi, xi * e1 * (1 - e2)), wt),
            ((xi, xi * e1 * (1 - e2)), (xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), wt),
        ]
    elif case == "edge":
        w1 = xi ** 3 * e1 ** 2
        w2 = xi ** 3 * e1 ** 2 * e2
        regions = [
            ((xi, xi * e1 * e3), (xi * (1 - e1 * e2), xi * e1 * (1 - e2)), w1),
            ((xi, xi * e1), (xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)), w2),
            ((xi * (1 - e1 * e2), xi * e1 * (1 - e2)), (xi, xi * e1 * e2 * e3), w2),
            ((xi * (1 - e1 * e2 * e3), xi * e1 * e2 * (1 - e3)), (xi, xi * e1), w2),
            ((xi * (1 - e1 * e2 * e3), xi * e1 * (1 - e2 * e3)), (xi, xi * e1 * e2), w2),
        ]
    elif case == "vert":
        wt = xi ** 3 * e2
        regions = [
            ((xi, xi * e1), (xi * e2, xi * e2 * e3), wt),
            ((xi * e2, xi * e2 * e3), (xi, xi * e1), wt),
        ]
    else:
        raise ValueError(case)
    xh = np.concatenate([np.stack(r[0], axis=1) for r in regions])
    yh = np.concatenate([np.stack(r[1], axis=1) for r in regions])
    w = np.concatenate([W * r[2] for r in regions])
    return xh, yh, w


def ref_to_bary(xh):
    """Reference point(s) of T^ -> barycentric (1 - x1, x1 - x2, x2)."""
    xh = np.atleast_2d(xh)
    return np.stack([1.0 - xh[:, 0], xh[:, 0] - xh[:, 1], xh[:, 1]], axis=1)
