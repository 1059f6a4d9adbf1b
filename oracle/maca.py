"""Multivariate adaptive cross approximation (Sec. 5.1, Alg. 2).

G (m x n x p) ~ sum_{t=1..r} C_t x_3 d_t (eq. summaca), built from r slices
and r fibres of G computed on demand by the `entry` call-backs.

Readings of the points the paper leaves open or states inconsistently:
* the first slice is frequency index 0 (the paper's k_1 = 0);
* the pivot (i, j) is the first maximum of |C_l| in row-major order;
* the next slice is the argmax of |d_l[k]| over slices not used yet (the
  paper's argmax would return the slice just used, where d_l = 1); ties go to
  the smallest k;
* the iteration stops on a zero pivot (|pivot| <= 1e-300), when all p slices
  are used, or when ||C_l||_F ||d_l||_2 <= eps ||G^(l)||_F, with the norm of
  G^(l) from the Gram identity of Sec. 5.1; every computed nonzero update is
  kept (the returned rank counts the update that met the stopping test).
"""
from __future__ import annotations

import numpy as np


def maca(entry_slice, entry_fibre, p: int, eps: float, max_rank: int | None = None):
    """Return (C, D, info): C (r, m, n) complex, D (p, r) complex.

    entry_slice(k) -> (m, n) slice G[:, :, k];
    entry_fibre(i, j) -> (p,) fibre G[i, j, :].
    """
    if max_rank is None:
        max_rank = p
    Cs, ds = [], []
    gram_c = np.zeros((0, 0), dtype=np.complex128)
    gram_d = np.zeros((0, 0), dtype=np.complex128)
    k = 0
    used = np.zeros(p, dtype=bool)
    pivots = []
    norm2 = 0.0
    while True:
        Cl = np.array(entry_slice(k), dtype=np.complex128)
        for Ct, dt in zip(Cs, ds):
            Cl = Cl - Ct * dt[k]
        a = np.abs(Cl)
        flat = int(np.argmax(a))
        i, j = divmod(flat, Cl.shape[1])
        piv = Cl[i, j]
        if not (abs(piv) > 1e-300):
            break
        fib = np.array(entry_fibre(i, j), dtype=np.complex128)
        for Ct, dt in zip(Cs, ds):
            fib = fib - Ct[i, j] * dt
        dl = fib / piv
        # Gram products for ||G^(l)||_F^2 (Sec. 5.1)
        gc_new = np.array([np.vdot(Ct, Cl) for Ct in Cs] + [np.vdot(Cl, Cl)])
        gd_new = np.array([np.vdot(dt, dl) for dt in ds] + [np.vdot(dl, dl)])
        n = len(Cs)
        G1 = np.zeros((n + 1, n + 1), dtype=np.complex128)
        G2 = np.zeros((n + 1, n + 1), dtype=np.complex128)
        G1[:n, :n] = gram_c
        G2[:n, :n] = gram_d
        G1[:, n] = gc_new
        G1[n, :] = np.conj(gc_new)
        G2[:, n] = gd_new
        G2[n, :] = np.conj(gd_new)
        gram_c, gram_d = G1, G2
        Cs.append(Cl)
        ds.append(dl)
        used[k] = True
        pivots.append((k, i, j))
        norm2 = float(np.real(np.sum(gram_c * gram_d)))
        upd = np.sqrt(np.real(gc_new[-1])) * np.sqrt(np.real(gd_new[-1]))
        if upd <= eps * np.sqrt(max(norm2, 0.0)) or len(Cs) >= max_rank or used.all():
            break
        cand = np.where(used, -1.0, np.abs(dl))
        k = int(np.argmax(cand))
    r = len(Cs)
    if r:
        C = np.stack(Cs)
        D = np.stack(ds, axis=1)
    else:
        C = np.zeros((0,) + np.shape(entry_slice(0)), dtype=np.complex128)
        D = np.zeros((p, 0), dtype=np.complex128)
    return C, D, {"rank": r, "pivots": pivots, "norm2": norm2}


def reconstruct(C, D):
    """G^(r)[i, j, k] = sum_t C[t, i, j] D[k, t]."""
    return np.einsum("tij,kt->ijk", C, D)
