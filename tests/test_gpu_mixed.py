"""Galerkin matrices with P1 functions for mixed boundary conditions on the
GPU (cqm_bem_p1_matrices: K with P1 trial functions, the adjoint double
layer K', the hypersingular operator D in Maue's form; Sec. 2.3 eq.
wavegalform, Sec. 3.2) against the oracle (oracle/mixed.py, pinned to the
sphere closed forms and a spherical wave), entry by entry at every solved
frequency, through host and device memory.
"""
import numpy as np
import pytest

from oracle import cqm, mixed
from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("level,N,dt", [(1, 24, 0.2), (2, 8, 0.1)])
def test_p1_matrices_equal_oracle(level, N, dt):
    from paper_2006_05186_gb300 import CqmBem, build
    build.build()
    m = synth.icosphere(level)
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", eta=1.0, cheb_m=4, n_min=32, aca_eps=1e-6)
    host = op.p1_matrices()
    dev = [t.cpu().numpy() for t in op.p1_matrices(device=True)]
    Ls = op.Ls
    op.close()
    s = cqm.frequencies(N, dt, 2)[:Ls]
    ref = mixed.p1_matrices(m.xyz, m.tri, s)
    for name, a, b, r in zip(("K1", "Kp", "D"), host, dev, ref):
        err = _rel(a, r)
        print(f"level {level}: {name} vs oracle {err:.2e}")
        assert err < 1e-10, (name, err)
        assert _rel(b, a) < 1e-13, name    # the device-memory outputs are the same sums
