"""Failure path of the bounded device waits (a status code, not a hang).

The tensor-core far coupling waits on mbarriers with a time limit.  Armed
from the host, its next launch makes one wait on a barrier that nothing
completes; the wait runs out after the handle's limit, the kernel drains what
it issued and returns, and the call reports CQM_ETIMEOUT.  The same handle
then solves correctly at the default limit.  Nothing here faults, traps or
waits without a limit.
"""
import numpy as np
import pytest

from oracle import dense
from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2006_05186_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_wait_expiry_is_reported_and_the_handle_recovers(lib):
    from paper_2006_05186_gb300 import CqmBem, CqmError, _lib
    m = synth.icosphere(3)
    N, dt = 32, 0.1
    p = synth.plane_wave_pulse()
    op = CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", aca_eps=1e-7)
    assert op.params.tensor_cores == 1
    b = op.rhs_plane_wave(p.direction, p.width, p.delay)
    q_ref = op.solve(b)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((op.Ls, m.nt)) + 1j * rng.standard_normal((op.Ls, m.nt))
    y_ref = op.apply_inner(x)

    op.set_wait_limit(2_000_000, expire_next=True)  # 2 ms
    with pytest.raises(CqmError) as ei:
        op.solve(b)
    assert ei.value.code == _lib.CQM_ETIMEOUT
    assert "wait expired" in str(ei.value) and "2000000 ns" in str(ei.value)
    op.set_wait_limit(0)
    q = op.solve(b)
    assert dense.rel_err(q, q_ref) <= 1e-12
    assert op.last_solve_info["max_rel_residual"] <= 1e-13

    op.set_wait_limit(1_000_000, expire_next=True)
    with pytest.raises(CqmError) as ei:
        op.apply_inner(x)
    assert ei.value.code == _lib.CQM_ETIMEOUT
    y = op.apply_inner(x)  # the probe is one-shot; the limit stays 1 ms
    assert np.array_equal(y, y_ref)
    op.close()


def test_wait_limit_arguments(lib):
    from paper_2006_05186_gb300 import _lib
    assert lib.cqm_bem_set_wait_limit(None, 10, 0) == _lib.CQM_EINVAL
