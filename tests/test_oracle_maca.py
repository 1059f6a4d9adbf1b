"""Pins of the MACA oracle (Sec. 5.1, Alg. 2, Thm. 3): exact low-rank tensors,
vanishing cross entries, the Gram-identity norm, geometric error decay."""
import numpy as np
import pytest

from oracle import cluster, cqm, h2, maca


def _lowrank(rng, m, n, p, r):
    C = rng.standard_normal((r, m, n)) + 1j * rng.standard_normal((r, m, n))
    d = rng.standard_normal((p, r)) + 1j * rng.standard_normal((p, r))
    return np.einsum("tij,kt->ijk", C, d)


@pytest.mark.parametrize("r", [1, 3, 6])
def test_T7_exact_rank_recovered(r):
    rng = np.random.default_rng(r)
    Gt = _lowrank(rng, 9, 7, 20, r)
    C, D, info = maca.maca(lambda k: Gt[:, :, k], lambda i, j: Gt[i, j, :], 20, 1e-10)
    assert info["rank"] in (r, r + 1)
    err = np.linalg.norm(maca.reconstruct(C, D) - Gt) / np.linalg.norm(Gt)
    assert err < 1e-13
    # the first r updates already reproduce the tensor
    err_r = np.linalg.norm(maca.reconstruct(C[:r], D[:, :r]) - Gt) / np.linalg.norm(Gt)
    assert err_r < 1e-12


def test_T7_cross_entries_vanish_and_gram_norm():
    rng = np.random.default_rng(11)
    Gt = _lowrank(rng, 8, 8, 15, 12) + 1e-3 * (rng.standard_normal((8, 8, 15)))
    C, D, info = maca.maca(lambda k: Gt[:, :, k], lambda i, j: Gt[i, j, :], 15, 1e-14, max_rank=6)
    Rs = Gt - maca.reconstruct(C, D)
    for (k, i, j) in info["pivots"]:
        assert np.max(np.abs(Rs[:, :, k])) < 1e-12 * np.max(np.abs(Gt))
        assert np.max(np.abs(Rs[i, j, :])) < 1e-12 * np.max(np.abs(Gt))
    explicit = np.linalg.norm(maca.reconstruct(C, D)) ** 2
    assert abs(info["norm2"] - explicit) < 1e-12 * explicit
    ks = [k for k, _, _ in info["pivots"]]
    assert ks[0] == 0 and len(set(ks)) == len(ks)


def test_rank_bounded_by_fibre_length():
    rng = np.random.default_rng(5)
    Gt = rng.standard_normal((6, 5, 4)) + 1j * rng.standard_normal((6, 5, 4))
    C, D, info = maca.maca(lambda k: Gt[:, :, k], lambda i, j: Gt[i, j, :], 4, 1e-16)
    assert info["rank"] <= 4
    assert np.linalg.norm(maca.reconstruct(C, D) - Gt) < 1e-12 * np.linalg.norm(Gt)


def test_T7_coupling_tensor_geometric_decay_and_tolerance():
    """Thm. 3: a far-field coupling tensor over the CQM frequencies is
    compressed with error ~ eps and the residual falls geometrically."""
    from paper_2006_05186_gb300 import synth
    m = synth.icosphere(3)
    t = cluster.build_tree(m.xyz, m.tri, 32)
    near, far = cluster.partition(t, 1.0)
    r, c = far[0]
    N = 64
    s = cqm.frequencies(N, 0.1, 2)[: cqm.n_solved(N + 1)]
    S = h2.coupling(t, r, c, s, 4)               # (L, 64, 64)
    Gt = np.moveaxis(S, 0, 2)
    errs = []
    for eps in (1e-2, 1e-4, 1e-6, 1e-8):
        C, D, info = maca.maca(lambda k: Gt[:, :, k], lambda i, j: Gt[i, j, :], Gt.shape[2], eps)
        e = np.linalg.norm(maca.reconstruct(C, D) - Gt) / np.linalg.norm(Gt)
        errs.append((info["rank"], e))
        assert e < 30 * eps, (eps, e)
    ranks = [x[0] for x in errs]
    assert ranks == sorted(ranks) and ranks[-1] < Gt.shape[2]


def test_maca_of_transposed_block_is_a_transposed_approximation():
    """Reading of the symmetric MACA: a block (c, r) of the symmetric single
    layer is the transpose of (r, c) at every frequency, and Alg. 2 run on the
    transposed tensor meets the same tolerance with the same rank (up to
    one); the transposed approximation of (r, c) is therefore as good an
    approximation of (c, r) as the one Alg. 2 computes for it."""
    from oracle import galerkin as G
    from paper_2006_05186_gb300 import synth
    m = synth.icosphere(2)
    t = cluster.build_tree(m.xyz, m.tri, 16)
    near, _ = cluster.partition(t, 1.0)
    r, c = next((r, c) for r, c in near if r != c)
    N, eps = 32, 1e-8
    s = cqm.frequencies(N, 0.1, 2)[: cqm.n_solved(N + 1)]
    ir, ic = t.indices(r), t.indices(c)
    I, J = np.meshgrid(ir, ic, indexing="ij")
    Gt = G.pair_entries(m.xyz, m.tri, I.ravel(), J.ravel(), s).reshape(len(ir), len(ic), -1)
    Gtt = np.transpose(Gt, (1, 0, 2))
    I2, J2 = np.meshgrid(ic, ir, indexing="ij")
    assert np.array_equal(G.pair_entries(m.xyz, m.tri, I2.ravel(), J2.ravel(), s).reshape(Gtt.shape), Gtt)
    C, D, info = maca.maca(lambda k: Gt[:, :, k], lambda i, j: Gt[i, j, :], len(s), eps)
    Ct, Dt, info_t = maca.maca(lambda k: Gtt[:, :, k], lambda i, j: Gtt[i, j, :], len(s), eps)
    assert abs(info["rank"] - info_t["rank"]) <= 1
    mirrored = np.transpose(maca.reconstruct(C, D), (1, 0, 2))
    nrm = np.linalg.norm(Gtt)
    assert np.linalg.norm(mirrored - Gtt) <= 20 * eps * nrm
    assert np.linalg.norm(maca.reconstruct(Ct, Dt) - Gtt) <= 20 * eps * nrm
