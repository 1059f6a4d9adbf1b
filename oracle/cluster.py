"""Cluster tree and block partition (Sec. 4.1, Defs. 2-4, eq. qadm).

Readings of what the paper leaves open:
* Geometric clustering: the box B_r is the tight axis-parallel box of the
  vertices of the triangles in r.  A cluster with #r <= n_min is a leaf.
  Otherwise split along the longest box side (ties: x before y before z) at
  the box midpoint (lo + hi) * 0.5; a triangle goes left iff its centroid
  ((P0 + P1) + P2) / 3 has that coordinate < midpoint.  If a side would be
  empty, split at the median instead: sort by (centroid coordinate, triangle
  index) and send the first floor(n/2) left.  Both sides keep the order of
  the parent (stable).
* Nodes are numbered breadth-first: by level, then by first position in the
  permutation.
* Admissibility on boxes (eq. qadm): diam = box diagonal, dist = Euclidean
  distance of the two boxes (0 when they overlap); r x c is admissible iff
  dist > 0 and max(diam_r, diam_c) <= eta * dist.  Sums of squares are formed
  in the order ((x^2 + y^2) + z^2).
* Block recursion exactly as Def. 3; admissible blocks form the far field,
  inadmissible leaf x leaf blocks the near field.  Lists are sorted by
  (row cluster, column cluster).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class ClusterTree:
    perm: np.ndarray          # (M,) triangle index at each position
    begin: np.ndarray         # (n_nodes,)
    end: np.ndarray           # (n_nodes,)
    lo: np.ndarray            # (n_nodes, 3)
    hi: np.ndarray            # (n_nodes, 3)
    son0: np.ndarray          # (n_nodes,) -1 for leaves
    son1: np.ndarray
    parent: np.ndarray
    level: np.ndarray
    sons: list = field(default_factory=list)

    @property
    def n_nodes(self):
        return len(self.begin)

    def is_leaf(self, r):
        return self.son0[r] < 0

    def indices(self, r):
        return self.perm[self.begin[r]:self.end[r]]


def centroids(xyz, tri):
    P = np.asarray(xyz, dtype=np.float64)[np.asarray(tri)]
    return (P[:, 0] + P[:, 1] + P[:, 2]) / 3.0


def build_tree(xyz, tri, n_min: int = 32) -> ClusterTree:
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri)
    M = len(tri)
    cen = centroids(xyz, tri)
    perm = np.arange(M, dtype=np.int64)
    nodes = []   # (begin, end, lo, hi, level, parent_tmp, sons_tmp)

    def rec(begin, end, level, parent):
        idx = perm[begin:end]
        V = xyz[tri[idx].ravel()]
        lo = V.min(axis=0)
        hi = V.max(axis=0)
        me = len(nodes)
        nodes.append([begin, end, lo, hi, level, parent, []])
        n = end - begin
        if n <= n_min:
            return me
        ext = hi - lo
        axis = int(np.argmax(ext))
        mid = (lo[axis] + hi[axis]) * 0.5
        left = cen[idx, axis] < mid
        nl = int(np.count_nonzero(left))
        if nl == 0 or nl == n:
            order = np.lexsort((idx, cen[idx, axis]))
            nl = n // 2
            left = np.zeros(n, dtype=bool)
            left[order[:nl]] = True
        perm[begin:end] = np.concatenate([idx[left], idx[~left]])
        a = rec(begin, begin + nl, level + 1, me)
        b = rec(begin + nl, end, level + 1, me)
        nodes[me][6] = [a, b]
        return me

    rec(0, M, 0, -1)
    # renumber breadth-first: by (level, begin)
    order = sorted(range(len(nodes)), key=lambda k: (nodes[k][4], nodes[k][0]))
    new_id = {old: new for new, old in enumerate(order)}
    n = len(nodes)
    begin = np.array([nodes[k][0] for k in order], dtype=np.int64)
    end = np.array([nodes[k][1] for k in order], dtype=np.int64)
    lo = np.array([nodes[k][2] for k in order])
    hi = np.array([nodes[k][3] for k in order])
    level = np.array([nodes[k][4] for k in order], dtype=np.int64)
    parent = np.array([new_id[nodes[k][5]] if nodes[k][5] >= 0 else -1 for k in order],
                      dtype=np.int64)
    son0 = -np.ones(n, dtype=np.int64)
    son1 = -np.ones(n, dtype=np.int64)
    sons = []
    for new, old in enumerate(order):
        s = [new_id[x] for x in nodes[old][6]]
        sons.append(s)
        if s:
            son0[new], son1[new] = s[0], s[1]
    return ClusterTree(perm, begin, end, lo, hi, son0, son1, parent, level, sons)


def box_diam(lo, hi):
    d = hi - lo
    return np.sqrt((d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2])


def box_dist(lo1, hi1, lo2, hi2):
    g = np.maximum(np.maximum(lo2 - hi1, lo1 - hi2), 0.0)
    return np.sqrt((g[..., 0] * g[..., 0] + g[..., 1] * g[..., 1]) + g[..., 2] * g[..., 2])


def admissible(t: ClusterTree, r: int, c: int, eta: float) -> bool:
    dr = box_diam(t.lo[r], t.hi[r])
    dc = box_diam(t.lo[c], t.hi[c])
    dist = box_dist(t.lo[r], t.hi[r], t.lo[c], t.hi[c])
    return bool(dist > 0.0 and max(dr, dc) <= eta * dist)


def partition(t: ClusterTree, eta: float):
    """(near, far): arrays of (row cluster, column cluster), sorted."""
    near, far = [], []
    stack = [(0, 0)]
    while stack:
        r, c = stack.pop()
        if admissible(t, r, c, eta):
            far.append((r, c))
            continue
        rl, cl = t.is_leaf(r), t.is_leaf(c)
        if rl and cl:
            near.append((r, c))
        elif rl:
            for c2 in t.sons[c]:
                stack.append((r, c2))
        elif cl:
            for r2 in t.sons[r]:
                stack.append((r2, c))
        else:
            for r2 in t.sons[r]:
                for c2 in t.sons[c]:
                    stack.append((r2, c2))
    near = np.array(sorted(near), dtype=np.int64).reshape(-1, 2)
    far = np.array(sorted(far), dtype=np.int64).reshape(-1, 2)
    return near, far
