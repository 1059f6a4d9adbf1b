"""Pins of the oracle's element rules: polynomial exactness and the in-plane
closed form of the Laplace potential of a flat triangle."""
import itertools
import math

import numpy as np
import pytest

from oracle import quadrature as Q


def _mono_exact(a, b):
    # int over T^ = {0 <= x2 <= x1 <= 1} of x1^a x2^b
    return 1.0 / ((b + 1) * (a + b + 2))


def _bary_rule_integral(bary, w, a, b):
    # reference coordinates from barycentric: x1 = 1 - l0, x2 = l2; area 1/2
    x1 = 1.0 - bary[:, 0]
    x2 = bary[:, 2]
    return 0.5 * np.sum(w * x1 ** a * x2 ** b)


def test_radon7_degree5_exact_and_not_degree6():
    assert abs(np.sum(Q.RADON7_W) - 1.0) < 1e-15
    for a in range(6):
        for b in range(6 - a):
            got = _bary_rule_integral(Q.RADON7_BARY, Q.RADON7_W, a, b)
            assert abs(got - _mono_exact(a, b)) < 1e-15
    errs = [abs(_bary_rule_integral(Q.RADON7_BARY, Q.RADON7_W, a, 6 - a) - _mono_exact(a, 6 - a))
            for a in range(7)]
    assert max(errs) > 1e-6


@pytest.mark.parametrize("g", [2, 3, 5])
def test_collapsed_rule_exactness(g):
    bary, w = Q.collapsed_rule(g)
    assert abs(np.sum(w) - 1.0) < 1e-14
    for a in range(2 * g - 1):
        for b in range(2 * g - 1 - a):
            got = _bary_rule_integral(bary, w, a, b)
            assert abs(got - _mono_exact(a, b)) < 1e-14 * max(1.0, 1 / _mono_exact(a, b))


@pytest.mark.parametrize("case", ["ident", "edge", "vert"])
def test_sauter_schwab_regions_partition_reference_square(case):
    """Every region set is a reparametrisation of T^ x T^: polynomials integrate exactly
    (g = 6 integrates the degree-11 pull-backs exactly)."""
    xh, yh, w = Q.sauter_schwab(case, 6)
    assert np.all(xh[:, 1] <= xh[:, 0] + 1e-15) and np.all(yh[:, 1] <= yh[:, 0] + 1e-15)
    assert np.all(xh >= -1e-15) and np.all(yh <= 1 + 1e-15)
    for a, b, c, d in itertools.product(range(3), repeat=4):
        got = np.sum(w * xh[:, 0] ** a * xh[:, 1] ** b * yh[:, 0] ** c * yh[:, 1] ** d)
        ref = _mono_exact(a, b) * _mono_exact(c, d)
        assert abs(got - ref) < 1e-13 * max(1.0, ref), (case, a, b, c, d)


def _chi(P, xh):
    return P[0][None, :] + xh[:, [0]] * (P[1] - P[0])[None, :] + xh[:, [1]] * (P[2] - P[1])[None, :]


def _area(P):
    return 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))


def laplace_potential_inplane(P, x):
    """int_T 1/|x - y| dy for points x in the plane of triangle T (closed form:
    sum over edges of h * (asinh(t_q/|h|) - asinh(t_p/|h|)), h the signed
    distance of x from the edge line, t_p, t_q the edge ends along the edge)."""
    n = np.cross(P[1] - P[0], P[2] - P[0])
    n /= np.linalg.norm(n)
    tot = np.zeros(len(x))
    for k in range(3):
        p, q = P[k], P[(k + 1) % 3]
        e = (q - p) / np.linalg.norm(q - p)
        mvec = np.cross(e, n)
        h = (p[None, :] - x) @ mvec
        tp = (p[None, :] - x) @ e
        tq = (q[None, :] - x) @ e
        ah = np.abs(h)
        safe = np.where(ah > 0, ah, 1.0)
        c = np.where(ah > 0, h * (np.arcsinh(tq / safe) - np.arcsinh(tp / safe)), 0.0)
        tot += c
    return tot


def _outer_rule(P, g):
    bary, w = Q.collapsed_rule(g)
    return bary @ P, _area(P) * w


def _ss_integral(Px, Py, case, g, kern):
    xh, yh, w = Q.sauter_schwab(case, g)
    r = np.linalg.norm(_chi(Px, xh) - _chi(Py, yh), axis=1)
    return 4 * _area(Px) * _area(Py) * np.sum(w * kern(r))


TAU = np.array([[0, 0, 0], [1, 0, 0], [0.3, 0.8, 0]], float)
COPLANAR = {
    "ident": TAU,
    "edge": np.array([[0, 0, 0], [1, 0, 0], [0.6, -0.7, 0]], float),
    "vert": np.array([[0, 0, 0], [-0.9, 0.2, 0], [-0.4, -0.8, 0]], float),
}


@pytest.mark.parametrize("case", ["ident", "edge", "vert"])
def test_sauter_schwab_laplace_closed_form(case):
    Pt = COPLANAR[case]
    xq, wq = _outer_rule(TAU, 60)
    ref = np.sum(wq * laplace_potential_inplane(Pt, xq))
    errs = {g: abs(_ss_integral(TAU, Pt, case, g, lambda r: 1 / r) - ref) / ref for g in (3, 5, 7)}
    assert errs[5] < 1e-6, errs
    assert errs[7] < errs[3], errs


def test_sauter_schwab_helmholtz_identical_vs_split():
    """exp(-sr)/r = 1/r + (exp(-sr)-1)/r: closed-form Laplace part plus a
    brute-force product rule on the bounded remainder; the brute force has a
    kink at x = y and converges algebraically toward the singular rule."""
    s = 2.0 + 3.0j
    xq, wq = _outer_rule(TAU, 60)
    lap = np.sum(wq * laplace_potential_inplane(TAU, xq))
    got = _ss_integral(TAU, TAU, "ident", 5, lambda rr: np.exp(-s * rr) / rr)
    errs = []
    for gb in (30, 60):
        xb, wb = _outer_rule(TAU, gb)
        r = np.linalg.norm(xb[:, None, :] - xb[None, :, :], axis=2)
        with np.errstate(invalid="ignore", divide="ignore"):
            rem = np.where(r > 0, (np.exp(-s * r) - 1.0) / np.where(r > 0, r, 1.0), -s)
        ref = lap + np.sum(wb[:, None] * wb[None, :] * rem)
        errs.append(abs(got - ref) / abs(ref))
    assert errs[1] < 1e-5 and errs[1] < errs[0] / 4, errs
