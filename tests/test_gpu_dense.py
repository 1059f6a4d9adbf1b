"""GPU parity of the dense FP64 path with the CPU oracle, through the C ABI.

Workload of the dense gate: the 320-triangle icosphere, BDF2, N = 32, dt = 0.1,
R = (1e-10)^(1/(2L)), Gaussian plane-wave pulse along +z, width 0.5, delay
from seed 20060518; tolerance 1e-10 relative (max over steps of the l2 error
over max step norm).  Smaller meshes, odd/even L, BDF1 and N = 1 are edge
cases of the same path.
"""
import numpy as np
import pytest

from oracle import cqm, dense, galerkin as G, incident
from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2006_05186_gb300 import build, _lib
    build.build()
    return _lib.load()


def _op(m, dt, N, bdf=2, **kw):
    from paper_2006_05186_gb300 import CqmBem
    return CqmBem(m.xyz, m.tri, dt, N, bdf, mode="dense", **kw)


@pytest.fixture(scope="module")
def c1(lib):
    """Dense GPU operator and oracle solution on the 320-triangle sphere."""
    m = synth.icosphere(2)
    N, dt = 32, 0.1
    p = synth.plane_wave_pulse()
    op = _op(m, dt, N)
    b_ref = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, p.delay)
    q_ref, info = dense.solve(m.xyz, m.tri, N, dt, 2, b_ref)
    yield dict(m=m, N=N, dt=dt, p=p, op=op, b_ref=b_ref, q_ref=q_ref, qhat_ref=info["qhat"])
    op.close()


def test_frequencies(c1):
    s = c1["op"].frequencies()
    ref = cqm.frequencies(c1["N"], c1["dt"], 2)
    assert np.max(np.abs(s - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_rhs_plane_wave(c1):
    p = c1["p"]
    b = c1["op"].rhs_plane_wave(p.direction, p.width, p.delay)
    assert np.max(np.abs(b - c1["b_ref"])) <= 1e-14 * np.max(np.abs(c1["b_ref"]))


def test_transforms(c1):
    op, N = c1["op"], c1["N"]
    R = cqm.default_R(N)
    rng = np.random.default_rng(1)
    b = rng.standard_normal((N + 1, op.M))
    g = op.forward_transform(b)
    g_ref = cqm.forward(b, R)[: op.Ls]
    assert np.max(np.abs(g - g_ref)) <= 1e-13 * np.max(np.abs(g_ref))
    back = op.inverse_transform(g)
    # inverse of the forward over all L frequencies: identity up to R^{-N} eps
    assert np.max(np.abs(back - b)) <= 1e-15 * R ** (-N) * (N + 1) * 10
    q_ref = cqm.inverse(np.concatenate([g_ref, np.conj(g_ref[1:(N + 1) - op.Ls + 1][::-1])]), R).real
    assert np.max(np.abs(back - q_ref)) <= 1e-15 * R ** (-N) * (N + 1) * 10


@pytest.mark.parametrize("N", [2048, 4095])
def test_transforms_long(lib, N):
    """The transforms keep their twiddle and R-power tables (24 L bytes) in
    shared memory, which exceeds the default 48 KB from L = 2049 on: long step
    counts (N = 2048 of the serving workload) still match the oracle."""
    m = synth.icosphere(0)
    op = _op(m, 0.05, N)
    R = cqm.default_R(N)
    rng = np.random.default_rng(7)
    b = rng.standard_normal((N + 1, op.M))
    g = op.forward_transform(b)
    g_ref = cqm.forward(b, R)[: op.Ls]
    assert np.max(np.abs(g - g_ref)) <= 1e-12 * np.max(np.abs(g_ref))
    back = op.inverse_transform(g)
    assert np.max(np.abs(back - b)) <= 1e-15 * R ** (-N) * (N + 1) * 10
    op.close()


def test_entries_every_case(c1):
    m, op = c1["m"], c1["op"]
    _, _, cen, diam = G.element_geometry(m.xyz, m.tri)
    rng = np.random.default_rng(2)
    I = rng.integers(0, m.nt, 3000)
    J = rng.integers(0, m.nt, 3000)
    I = np.concatenate([I, np.arange(m.nt)[:40]])
    J = np.concatenate([J, np.arange(m.nt)[:40]])
    # add pairs of every singular/near class
    A, B = np.meshgrid(np.arange(60), np.arange(m.nt), indexing="ij")
    case = G.classify(m.tri, A.ravel(), B.ravel(), cen, diam, G.QuadParams())
    for c in range(5):
        sel = np.nonzero(case == c)[0][:50]
        I = np.concatenate([I, A.ravel()[sel]])
        J = np.concatenate([J, B.ravel()[sel]])
    freq = np.array([0, 3, 16, 17, 31, 32])
    s = cqm.frequencies(c1["N"], c1["dt"], 2)
    got = op.entries(I, J, freq)
    ref = G.pair_entries(m.xyz, m.tri, I, J, s[freq])
    err = np.max(np.abs(got - ref) / np.abs(ref))
    assert err < 1e-12, err


def test_dense_apply(c1):
    m, op, N = c1["m"], c1["op"], c1["N"]
    s = cqm.frequencies(N, c1["dt"], 2)[: op.Ls]
    V = G.dense_matrices(m.xyz, m.tri, s[[0, 7, op.Ls - 1]])
    rng = np.random.default_rng(3)
    x = rng.standard_normal((op.Ls, op.M)) + 1j * rng.standard_normal((op.Ls, op.M))
    y = op.apply(x)
    for k, l in enumerate([0, 7, op.Ls - 1]):
        ref = V[k] @ x[l]
        assert np.max(np.abs(y[l] - ref)) <= 1e-13 * np.max(np.abs(ref))
    # device memory path gives the same numbers
    yd = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(yd, y)


def test_solve_frequencies(c1):
    op = c1["op"]
    g = op.forward_transform(c1["b_ref"])
    q, info = op.solve_frequencies(g)
    assert info["converged"] == op.Ls and info["max_rel_residual"] <= 1e-13
    ref = c1["qhat_ref"][: op.Ls]
    err = np.max(np.linalg.norm(q - ref, axis=1) / np.linalg.norm(ref, axis=1))
    assert err < 1e-11, err


def test_C1_dense_solve_gate(c1):
    """The dense FP64 gate: <= 1e-10 relative to the oracle, host and device buffers."""
    op = c1["op"]
    q = op.solve(c1["b_ref"])
    err = dense.rel_err(q, c1["q_ref"])
    assert err <= 1e-10, err
    qd = op.solve(torch.from_numpy(c1["b_ref"]).cuda()).cpu().numpy()
    assert dense.rel_err(qd, c1["q_ref"]) <= 1e-10
    assert op.last_solve_info["converged"] == op.Ls


@pytest.mark.parametrize("shape,N,bdf,dt", [
    ("tetra", 1, 2, 0.2),        # L = 2 (even), Ls = 2
    ("octa", 2, 1, 0.2),         # L = 3, BDF1
    ("ico0", 7, 2, 0.15),        # L = 8 (even), Ls = 5
    ("ico1", 9, 1, 0.3),         # ragged M = 80
    ("ellip1", 12, 2, 0.1),
])
def test_dense_edge_cases(lib, shape, N, bdf, dt):
    m = {"tetra": synth.tetrahedron, "octa": synth.octahedron, "ico0": lambda: synth.icosphere(0),
         "ico1": lambda: synth.icosphere(1),
         "ellip1": lambda: synth.ellipsoid(1, (0.6, 1.0, 1.7))}[shape]()
    p = synth.plane_wave_pulse(width=0.4)
    delay = 1.0
    # small L means small R = (1e-10)^(1/(2L)): the inverse transform scales
    # per-frequency rounding by up to R^-N (2.4e4 at N = 7), so these cases
    # iterate to the FP64 floor instead of the default 1e-13
    op = _op(m, dt, N, bdf, gmres_tol=1e-15, gmres_max_iter=400)
    b = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, delay)
    q = op.solve(b, allow_noconv=True)
    q_ref, _ = dense.solve(m.xyz, m.tri, N, dt, bdf, b)
    op.close()
    assert dense.rel_err(q, q_ref) <= 1e-10


def test_zero_rhs_gives_zero(lib):
    m = synth.icosphere(0)
    op = _op(m, 0.1, 6)
    q = op.solve(np.zeros((7, m.nt)))
    op.close()
    assert np.all(q == 0.0)
