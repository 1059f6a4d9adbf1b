"""The oracle's H^2-expanded matrices and per-frequency solves, evaluated over
a process pool.  TEST INFRASTRUCTURE ONLY (see the package docstring).

Nothing here adds arithmetic: every near-field entry is `galerkin.pair_entries`
of its pair and every far block is `U_r S_b(s_l) U_c^T` exactly as in
`h2.h2_matrices` (eq. uniformlr); the pool only evaluates independent pairs
and blocks in different processes, so the result equals the serial
`h2.h2_matrices` bit for bit (checked by a CPU test).  The per-frequency solve
is LAPACK's LU (numpy.linalg.solve), one frequency at a time, as in
`dense.solve_frequencies`.

Workers are started with the `spawn` method (a forked child of a process that
has initialised CUDA can hang) and with one BLAS thread each.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from contextlib import contextmanager

import numpy as np

from . import h2
from .galerkin import QuadParams, pair_entries

_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


@contextmanager
def _pool(workers: int):
    """A spawn pool whose workers run single-threaded BLAS."""
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    for k in _THREAD_VARS:
        os.environ[k] = "1"
    try:
        pool = mp.get_context("spawn").Pool(workers)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    try:
        yield pool
    finally:
        pool.close()
        pool.join()


def default_workers() -> int:
    """The host cores this process may run on (its affinity mask)."""
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 1
    return max(1, min(64, n))


def _near_chunk(args):
    xyz, tri, I, J, s, qp = args
    return pair_entries(xyz, tri, I, J, s, qp)


def _far_chunk(args):
    xyz, tri, tree, blocks, s, m = args
    cache = {}

    def U(r):
        if r not in cache:
            cache[r] = h2.cluster_basis(xyz, tri, tree, r, m)
        return cache[r]

    out = []
    for r, c in blocks:
        S = h2.coupling(tree, r, c, s, m)
        out.append((U(r) @ S) @ U(c).T)
    return out


def h2_matrices(xyz, tri, s, tree, near, far, m: int, qp: QuadParams = QuadParams(),
                workers: int | None = None):
    """Same result as `h2.h2_matrices` (len(s), M, M), evaluated over a pool."""
    s = np.atleast_1d(np.asarray(s, dtype=np.complex128))
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri)
    M = len(tri)
    workers = workers or default_workers()
    out = np.zeros((len(s), M, M), dtype=np.complex128)
    I, J = [], []
    for r, c in near:
        a, b = np.meshgrid(tree.indices(r), tree.indices(c), indexing="ij")
        I.append(a.ravel())
        J.append(b.ravel())
    I = np.concatenate(I) if I else np.zeros(0, np.int64)
    J = np.concatenate(J) if J else np.zeros(0, np.int64)
    nchunk = 4 * workers
    near_parts = [(xyz, tri, Ii, Jj, s, qp)
                  for Ii, Jj in zip(np.array_split(I, nchunk), np.array_split(J, nchunk)) if len(Ii)]
    far = [tuple(map(int, b)) for b in far]
    far_parts = [(xyz, tri, tree, [far[k] for k in ks], s, m)
                 for ks in np.array_split(np.arange(len(far)), nchunk) if len(ks)]
    with _pool(workers) as pool:
        near_res = pool.map_async(_near_chunk, near_parts)
        far_res = pool.map_async(_far_chunk, far_parts)
        for (_, _, Ii, Jj, _, _), e in zip(near_parts, near_res.get()):
            out[:, Ii, Jj] = e.T
        for part, blks in zip(far_parts, far_res.get()):
            for (r, c), blk in zip(part[3], blks):
                out[:, tree.indices(r)[:, None], tree.indices(c)[None, :]] = blk
    return out


def h2_solve_frequencies(xyz, tri, s, tree, near, far, m: int, ghat,
                         qp: QuadParams = QuadParams(), workers: int | None = None):
    """qhat_l = V_l^{-1} ghat_l with the H^2-expanded V_l of each frequency in s
    (ghat: (len(s), M)); one LAPACK LU per frequency."""
    V = h2_matrices(xyz, tri, s, tree, near, far, m, qp, workers)
    return np.stack([np.linalg.solve(V[k], ghat[k]) for k in range(len(V))])
