"""GPU parity of the compressed path (H^2 far field + frequency MACA) with the
CPU oracle, through the C ABI.

* cluster tree and partition: bit-exact against the oracle (same readings of
  Defs. 2-4 and eq. qadm);
* the compressed operator with a tight MACA tolerance reproduces the oracle's
  H^2-expanded matrices (Chebyshev interpolation, no frequency compression);
* MACA factors of sampled blocks approximate the exact block tensors to the
  stated tolerance;
* the compressed solve matches the H^2-expanded oracle solve (time domain on
  1280 triangles; the 5120-triangle, N = 256 workload is in test_gpu_headline).
"""
import numpy as np
import pytest

from oracle import cluster, cqm, dense, galerkin as G, h2, incident, maca, pool
from paper_2006_05186_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2006_05186_gb300 import build, _lib
    build.build()
    return _lib.load()


def _op(m, dt, N, **kw):
    from paper_2006_05186_gb300 import CqmBem
    return CqmBem(m.xyz, m.tri, dt, N, 2, mode="h2maca", **kw)


MESHES = {
    "sphere320": lambda: synth.icosphere(2),
    "sphere1280": lambda: synth.icosphere(3),
    "sphere5120": lambda: synth.icosphere(4),
    "torus1280": lambda: synth.torus_for(1280),
    "ellipsoid320": lambda: synth.ellipsoid(2, (0.5, 1.0, 2.0)),
    "cube1280": lambda: synth.rounded_cube(3),
}


@pytest.mark.parametrize("name", list(MESHES))
def test_tree_and_partition_bit_exact(lib, name):
    m = MESHES[name]()
    op = _op(m, 0.1, 4, rank_cap=3)
    t_ref = cluster.build_tree(m.xyz, m.tri, 32)
    near_ref, far_ref = cluster.partition(t_ref, 1.0)
    t = op.tree()
    assert np.array_equal(t["perm"], t_ref.perm)
    assert np.array_equal(t["begin"], t_ref.begin) and np.array_equal(t["end"], t_ref.end)
    assert np.array_equal(t["son0"], t_ref.son0) and np.array_equal(t["son1"], t_ref.son1)
    assert np.array_equal(t["level"], t_ref.level)
    assert np.array_equal(t["lo"], t_ref.lo) and np.array_equal(t["hi"], t_ref.hi)
    blk = op.blocks()
    assert np.array_equal(blk["near"], near_ref) and np.array_equal(blk["far"], far_ref)
    op.close()


def _h2_reference(m, N, dt, freqs, tree_ref, near, far, cheb_m=4):
    s = cqm.frequencies(N, dt, 2)[freqs]
    return pool.h2_matrices(m.xyz, m.tri, s, tree_ref, near, far, cheb_m)


@pytest.mark.parametrize("cheb_m", [4, 3, 2])
def test_apply_tight_eps_equals_h2_expanded(lib, cheb_m):
    """The FP64 apply equals the oracle's H^2-expanded matrices (MACA at a
    tolerance below rounding) to 1e-10, and the FP32 inner operator to FP32
    accuracy, for every supported number m of Chebyshev points per axis."""
    m = synth.icosphere(3)
    N, dt = 16, 0.1
    op = _op(m, dt, N, aca_eps=1e-14, rank_cap=64, cheb_m=cheb_m)
    t_ref = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t_ref, 1.0)
    Ls = op.Ls
    V = _h2_reference(m, N, dt, np.arange(Ls), t_ref, near, far, cheb_m)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((Ls, m.nt)) + 1j * rng.standard_normal((Ls, m.nt))
    y = op.apply(x)
    yi = op.apply_inner(x)
    for l in range(Ls):
        ref = V[l] @ x[l]
        err = np.linalg.norm(y[l] - ref) / np.linalg.norm(ref)
        assert err < 1e-10, (l, err)
        err_i = np.linalg.norm(yi[l] - ref) / np.linalg.norm(ref)
        assert err_i < 1e-5, (l, err_i)
    op.close()


def test_maca_blocks_meet_tolerance(lib):
    m = synth.icosphere(3)
    N, dt, eps = 64, 0.1, 1e-6
    op = _op(m, dt, N, aca_eps=eps)
    t_ref = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t_ref, 1.0)
    s = cqm.frequencies(N, dt, 2)[: op.Ls]
    blk = op.blocks()
    rng = np.random.default_rng(5)
    for b in rng.choice(len(near), 6, replace=False):
        r, c = near[b]
        ir, ic = t_ref.indices(r), t_ref.indices(c)
        I, J = np.meshgrid(ir, ic, indexing="ij")
        Gt = G.pair_entries(m.xyz, m.tri, I.ravel(), J.ravel(), s).reshape(len(ir), len(ic), -1)
        Cg, Dg = op.block_factors(0, int(b))
        approx = np.einsum("tij,tk->ijk", Cg, Dg)
        err = np.linalg.norm(approx - Gt) / np.linalg.norm(Gt)
        assert err < 10 * eps, (b, err)
        _, _, info = maca.maca(lambda k: Gt[:, :, k], lambda i, j: Gt[i, j, :], len(s), eps)
        assert abs(blk["near_rank"][b] - info["rank"]) <= 2
    for b in rng.choice(len(far), 10, replace=False):
        r, c = far[b]
        St = np.moveaxis(h2.coupling(t_ref, r, c, s, 4), 0, 2)
        Cg, Dg = op.block_factors(1, int(b))
        approx = np.einsum("tij,tk->ijk", Cg, Dg)
        err = np.linalg.norm(approx - St) / np.linalg.norm(St)
        assert err < 10 * eps, (b, err)
        _, _, info = maca.maca(lambda k: St[:, :, k], lambda i, j: St[i, j, :], len(s), eps)
        assert abs(blk["far_rank"][b] - info["rank"]) <= 2
    op.close()


@pytest.fixture(scope="module")
def ref1280():
    m = synth.icosphere(3)
    N, dt = 32, 0.1
    p = synth.plane_wave_pulse()
    from oracle import incident
    b = incident.rhs_plane_wave(m.xyz, m.tri, N, dt, p.direction, p.width, p.delay)
    t_ref = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t_ref, 1.0)
    q_ref, _ = dense.solve(m.xyz, m.tri, N, dt, 2, b,
                           matrices=lambda ss: pool.h2_matrices(m.xyz, m.tri, ss, t_ref, near, far, 4))
    return dict(m=m, N=N, dt=dt, b=b, q_ref=q_ref)


@pytest.mark.parametrize("eps,tol", [(1e-7, 1e-6), (1e-6, 1e-5)])
def test_compressed_solve_time_domain_1280(lib, ref1280, eps, tol):
    """Time-domain gate against the H^2-expanded oracle (no MACA) at 1280
    triangles.  The MACA tolerance bounds the operator error per block; the
    solution error is that times the conditioning, so the 1e-6 solution gate
    is met with eps = 1e-7 and eps = 1e-6 gives ~kappa * 1e-6."""
    r = ref1280
    op = _op(r["m"], r["dt"], r["N"], aca_eps=eps)
    q = op.solve(r["b"])
    err = dense.rel_err(q, r["q_ref"])
    print(f"eps={eps}: time-domain rel err vs H2-expanded oracle {err:.3e}")
    assert err <= tol, err
    op.close()


@pytest.mark.parametrize("precond,inner_fp32,tensor_cores",
                         [(0, 0, 1), (1, 0, 1), (0, 1, 1), (1, 1, 1), (1, 1, 2), (1, 1, 0)])
def test_solver_variants_agree(lib, precond, inner_fp32, tensor_cores):
    """Preconditioning and the FP32 inner operator change the iteration, not
    the answer: every variant meets the FP64 residual target and agrees with
    the plain FP64 solve to ~1e-10 in the time domain."""
    m = synth.icosphere(3)
    N, dt = 32, 0.1
    p = synth.plane_wave_pulse()
    ref_op = _op(m, dt, N, precond=0, inner_fp32=0)
    b = ref_op.rhs_plane_wave(p.direction, p.width, p.delay)
    q_ref = ref_op.solve(b)
    ref_op.close()
    op = _op(m, dt, N, precond=precond, inner_fp32=inner_fp32, tensor_cores=tensor_cores)
    q = op.solve(b)
    info = op.last_solve_info
    op.close()
    assert info["converged"] == N // 2 + 1 and info["max_rel_residual"] <= 1e-13
    assert dense.rel_err(q, q_ref) <= 1e-10


def test_point_cache_matches_direct_quadrature(lib):
    """Cached near-field quadrature points give the MACA factors of the
    direct quadrature (same pivots and ranks, entries equal to rounding)."""
    m = synth.icosphere(3)
    N, dt = 24, 0.1
    a = _op(m, dt, N, cache_quadrature=1, maca_ff=0)
    b = _op(m, dt, N, cache_quadrature=0)
    ba, bb = a.blocks(), b.blocks()
    assert np.array_equal(ba["near_rank"], bb["near_rank"])
    assert np.array_equal(ba["far_rank"], bb["far_rank"])
    rng = np.random.default_rng(9)
    for k in rng.choice(len(ba["near"]), 20, replace=False):
        Ca, Da = a.block_factors(0, int(k))
        Cb, Db = b.block_factors(0, int(k))
        ta = np.einsum("tij,tk->ijk", Ca, Da)
        tb = np.einsum("tij,tk->ijk", Cb, Db)
        assert np.linalg.norm(ta - tb) <= 1e-12 * np.linalg.norm(tb)
    a.close()
    b.close()


@pytest.mark.parametrize("tensor_cores", [0, 1, 2])
def test_inner_operator_fp32_accuracy(lib, tensor_cores):
    """The inner operator (FP32 SIMT; bf16 or TF32 tensor cores with the
    hi/lo three-product split) agrees with the FP64-accurate apply to 1e-5,
    frequency by frequency (N = 40: one padded 128-frequency chunk)."""
    m = synth.icosphere(4)
    N, dt = 40, 0.1
    op = _op(m, dt, N, tensor_cores=tensor_cores)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((op.Ls, m.nt)) + 1j * rng.standard_normal((op.Ls, m.nt))
    y = op.apply(x)
    yi = op.apply_inner(x)
    op.close()
    err = np.linalg.norm(yi - y, axis=1) / np.linalg.norm(y, axis=1)
    # the three-product split keeps ~17 (bf16) or ~21 (TF32) bits per operand;
    # a wrong fragment layout would give errors of order one
    print(f"tensor_cores={tensor_cores}: max per-frequency error {np.max(err):.2e}")
    assert np.max(err) < 1e-5, err


def test_single_product_terms(lib):
    """The trailing rank terms that take one bf16 product (tc_single_ratio,
    default 1e-3 of the largest far term per frequency) leave the inner
    operator as accurate as the three-product split throughout, frequency by
    frequency; with the ratio 0 no term takes it."""
    m = synth.icosphere(4)
    N, dt = 40, 0.1
    rng = np.random.default_rng(13)
    x = None
    err, single = {}, {}
    for ratio in (0.0, None):
        kw = {} if ratio is None else {"tc_single_ratio": ratio}
        op = _op(m, dt, N, aca_eps=1e-9, **kw)
        if x is None:
            x = rng.standard_normal((op.Ls, m.nt)) + 1j * rng.standard_normal((op.Ls, m.nt))
        y = op.apply(x)
        yi = op.apply_inner(x)
        single[ratio] = op.info()["tc_single_terms"]
        total = op.info()["rank_sum_far"]
        op.close()
        err[ratio] = np.linalg.norm(yi - y, axis=1) / np.linalg.norm(y, axis=1)
    print(f"single-product terms {single[None]} of {total}; max error {np.max(err[0.0]):.2e} (three "
          f"products) {np.max(err[None]):.2e} (trailing terms single)")
    assert single[0.0] == 0 and total // 10 < single[None] < total
    assert np.max(err[None]) < 1e-5 and np.all(err[None] <= 2.0 * err[0.0] + 1e-7)


def test_expanded_near_field_equals_factored(lib):
    """The near field and the far couplings expanded per frequency
    (sum_t C_t d_t, near in FP64, far in float-float) are the factored
    operator up to rounding: the FP64-accurate applies agree to 1e-12, and
    the FP32 inner operator of the expanded near field is at least as close
    to the FP64 operator as the factored FP32 one (its entries are rounded
    once)."""
    m = synth.icosphere(3)
    N, dt = 64, 0.1
    ops = {e: _op(m, dt, N, expand_near=e, expand_far=e) for e in (0, 1)}
    assert ops[1].info()["device_bytes"] > ops[0].info()["device_bytes"]
    Ls = ops[0].Ls
    rng = np.random.default_rng(11)
    x = rng.standard_normal((Ls, m.nt)) + 1j * rng.standard_normal((Ls, m.nt))
    y = {e: ops[e].apply(x) for e in (0, 1)}
    yi = {e: ops[e].apply_inner(x) for e in (0, 1)}
    for l in range(Ls):
        nrm = np.linalg.norm(y[0][l])
        assert np.linalg.norm(y[1][l] - y[0][l]) <= 1e-12 * nrm, l
        e_fact = np.linalg.norm(yi[0][l] - y[0][l]) / nrm
        e_exp = np.linalg.norm(yi[1][l] - y[1][l]) / nrm
        assert e_exp <= 1e-5 and e_exp <= 2.0 * e_fact + 1e-7, (l, e_exp, e_fact)
    for op in ops.values():
        op.close()


@pytest.mark.parametrize("maca_ff", [1, 0])
def test_maca_full_rank_reproduces_entries(lib, maca_ff):
    """With every solved frequency taken as a slice, the MACA reproduces the
    block tensors exactly; the float-float (maca_ff = 1) and FP64 slice and
    fibre evaluations both match the oracle's entries and Chebyshev
    couplings to 1e-11 at 33 frequencies up to |s| = 40."""
    m = synth.icosphere(3)
    N, dt = 64, 0.1
    op = _op(m, dt, N, aca_eps=1e-15, rank_cap=33, maca_ff=maca_ff)
    t_ref = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t_ref, 1.0)
    s = cqm.frequencies(N, dt, 2)[: op.Ls]
    rng = np.random.default_rng(21)
    worst = 0.0
    for b in rng.choice(len(near), 12, replace=False):
        r, c = near[b]
        ir, ic = t_ref.indices(r), t_ref.indices(c)
        I, J = np.meshgrid(ir, ic, indexing="ij")
        Gt = G.pair_entries(m.xyz, m.tri, I.ravel(), J.ravel(), s).reshape(len(ir), len(ic), -1)
        Cg, Dg = op.block_factors(0, int(b))
        worst = max(worst, np.linalg.norm(np.einsum("tij,tk->ijk", Cg, Dg) - Gt) / np.linalg.norm(Gt))
    for b in rng.choice(len(far), 12, replace=False):
        r, c = far[b]
        St = np.moveaxis(h2.coupling(t_ref, r, c, s, 4), 0, 2)
        Cg, Dg = op.block_factors(1, int(b))
        worst = max(worst, np.linalg.norm(np.einsum("tij,tk->ijk", Cg, Dg) - St) / np.linalg.norm(St))
    op.close()
    print(f"maca_ff={maca_ff}: worst block error {worst:.2e}")
    assert worst <= 1e-11, worst


def test_maca_ff_matches_fp64_maca(lib):
    """The float-float slices and fibres change the MACA's entries only at
    rounding level: the ranks agree to one and the two compressed operators
    agree to a few times the MACA tolerance at every frequency."""
    m = synth.icosphere(3)
    N, dt, eps = 64, 0.1, 1e-9
    a = _op(m, dt, N, aca_eps=eps, maca_ff=1)
    b = _op(m, dt, N, aca_eps=eps, maca_ff=0)
    ba, bb = a.blocks(), b.blocks()
    assert np.max(np.abs(ba["near_rank"] - bb["near_rank"])) <= 1
    assert np.max(np.abs(ba["far_rank"] - bb["far_rank"])) <= 1
    rng = np.random.default_rng(5)
    x = rng.standard_normal((a.Ls, m.nt)) + 1j * rng.standard_normal((a.Ls, m.nt))
    ya, yb = a.apply(x), b.apply(x)
    err = np.linalg.norm(ya - yb, axis=1) / np.linalg.norm(yb, axis=1)
    a.close()
    b.close()
    assert np.max(err) <= 20 * eps, err
