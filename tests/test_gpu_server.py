"""Many scattering problems on one GPU through the request server
(cqm_server_create, cqm_bem_submit, cqm_bem_poll).

* A mixed batch (sphere, ellipsoid, rounded cube, torus; 320 to 1280
  triangles; N from 32 to 128; dt = 0.4 times the mean edge length) runs on
  three workers whose kernels overlap; every result equals the same problem
  solved alone with the same parameters, and every result is within 1e-6 of
  the oracle in the time domain (LU of the H^2-expanded V_l at every solved
  frequency; MACA tolerance 1e-9).
* A request whose estimated footprint exceeds the server's budget is refused
  with CQM_ENOMEM at submit, and a budget that holds one request at a time
  runs the requests one at a time.
"""
import time

import numpy as np
import pytest

from oracle import cluster, cqm, dense, incident, pool
from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EPS = 1e-9


def _batch():
    out = []
    for k, (shape, level, N) in enumerate([("sphere", 2, 32), ("ellipsoid", 3, 64), ("cube", 2, 128),
                                             ("torus", 1280, 64), ("sphere", 3, 48)]):
        if shape == "sphere":
            m = synth.icosphere(level)
        elif shape == "ellipsoid":
            m = synth.ellipsoid(level, (0.6, 1.0, 1.7))
        elif shape == "cube":
            m = synth.rounded_cube(level)
        else:
            m = synth.torus_for(level)
        p = synth.plane_wave_pulse(seed=synth.SEED_BASE + 100 + k, width=0.4 + 0.1 * k)
        out.append(dict(m=m, N=N, dt=0.4 * synth.mean_edge_length(m), p=p))
    return out


def _oracle(m, N, dt, p):
    L = N + 1
    R = cqm.default_R(N)
    t = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t, 1.0)
    b = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, p.delay)
    g = cqm.forward(b, R)
    s = cqm.frequencies(N, dt, 2)
    Ls = L // 2 + 1
    qh = pool.h2_solve_frequencies(m.xyz, m.tri, s[:Ls], t, near, far, 4, g[:Ls], workers=8)
    return cqm.inverse(dense.fill_conjugate(qh, L), R).real


def test_batch_equals_alone_and_oracle():
    from paper_2006_05186_gb300 import CqmBem, Server, build
    build.build()
    batch = _batch()
    srv = Server(workers=3)
    tickets = [srv.submit(c["m"].xyz, c["m"].tri, c["dt"], c["N"], direction=c["p"].direction,
                          width=c["p"].width, delay=c["p"].delay, aca_eps=EPS) for c in batch]
    results = [srv.poll(t) for t in tickets]
    srv.close()
    workers = set()
    for c, (code, q, info) in zip(batch, results):
        assert code == 0, info
        workers.add(info["worker"])
        assert info["solve"]["converged"] == c["N"] // 2 + 1
        assert info["device_bytes"] <= info["bytes_estimate"]
        op = CqmBem(c["m"].xyz, c["m"].tri, c["dt"], c["N"], 2, aca_eps=EPS, expand_far=0)
        b = op.rhs_plane_wave(c["p"].direction, c["p"].width, c["p"].delay)
        q_alone = op.solve(b)
        op.close()
        e_alone = dense.rel_err(q, q_alone)
        e_oracle = dense.rel_err(q, _oracle(c["m"], c["N"], c["dt"], c["p"]))
        print(f"M={c['m'].nt} N={c['N']}: alone vs batched {e_alone:.1e}, vs oracle {e_oracle:.2e}, "
              f"queue {info['t_queue_ms']:.0f} ms, worker {info['worker']}")
        assert e_alone <= 1e-12
        assert e_oracle <= 1e-6
    assert len(workers) > 1


def test_over_budget_request_is_refused():
    from paper_2006_05186_gb300 import CqmError, Server, _lib, build, estimate_bytes
    build.build()
    m = synth.icosphere(4)
    need = estimate_bytes(m.nt, 256, expand_far=0)
    srv = Server(workers=1, byte_budget=need // 2)
    with pytest.raises(CqmError) as ei:
        srv.submit(m.xyz, m.tri, 0.1, 256)
    assert ei.value.code == _lib.CQM_ENOMEM
    srv.close()


def test_budget_for_one_request_runs_them_one_at_a_time():
    from paper_2006_05186_gb300 import Server, build, estimate_bytes
    build.build()
    m = synth.icosphere(3)
    need = estimate_bytes(m.nt, 64, expand_far=0)
    srv = Server(workers=3, byte_budget=int(need * 1.5))
    tickets = [srv.submit(m.xyz, m.tri, 0.1, 64) for _ in range(3)]
    peak = 0
    pending = set(tickets)
    done = {}
    while pending:
        peak = max(peak, srv.load()["running"])
        for t in list(pending):
            code, q, info = srv.poll(t, wait=False)
            if q is not None:
                done[t] = (code, q)
                pending.discard(t)
        time.sleep(0.001)
    srv.close()
    assert peak == 1
    qs = [done[t][1] for t in tickets]
    assert all(done[t][0] == 0 for t in tickets)
    assert all(np.array_equal(qs[0], q) for q in qs[1:])
